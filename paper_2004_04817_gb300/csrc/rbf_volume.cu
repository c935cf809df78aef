// rbf_volume.cu -- volume displacement sum (Eq. 6 of arXiv:2004.04817):
//     dv_v = sum_{j in S} w_j phi(|x_v - r_j| / R),  v = 1..N_v.
//
// FP32 kernel: every thread owns 4 volume points (coordinates pre-scaled by
// 1/R) in paired registers, centres and weights are staged in shared memory
// in tiles and read as broadcasts, so a pair costs ~16 FP32-pipe
// instructions including one MUFU square root and no memory traffic.
// Double-float kernel: the same structure with every value an unevaluated
// sum of two floats (~110 FP32-pipe instructions per pair, FP64-level
// results).  FP64 kernel: the same structure in double precision (reference
// arithmetic).  The traffic is the packed points: the kernels are bound by
// the FP32 pipe.
#include <algorithm>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kVolThreads = 256;
constexpr int kVolP = 2;               // paired registers per thread (4 points)
constexpr int kTileF32 = 2048;         // centres per shared-memory tile (96 KB)
constexpr int kTileF64 = 1024;         // centres per shared-memory tile (64 KB)
constexpr int kTileFF = 1024;          // double-float centres per tile (64 KB)
constexpr int kVolQFF = 2;             // points per thread, double-float kernel

// ---------------------------------------------------------------------------
// Packing: FP64 row-major inputs -> scaled, vector-aligned device layouts.
// ---------------------------------------------------------------------------
__global__ void k_pack_points_f32(const double *__restrict__ x, int64_t n, double inv_r,
                                  float4 *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = make_float4((float)(x[3 * i] * inv_r), (float)(x[3 * i + 1] * inv_r),
                             (float)(x[3 * i + 2] * inv_r), 0.0f);
    }
}

// grid-split points (x / R) for the double-float kernels
__global__ void k_pack_points_ff(const double *__restrict__ x, int64_t n, double inv_r,
                                 const unsigned long long *__restrict__ gmax,
                                 float4 *__restrict__ hi, float4 *__restrict__ lo)
{
    const double G = grid_of(gmax);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h0, l0, h1, l1, h2, l2;
        split_grid(x[3 * i] * inv_r, G, h0, l0);
        split_grid(x[3 * i + 1] * inv_r, G, h1, l1);
        split_grid(x[3 * i + 2] * inv_r, G, h2, l2);
        hi[i] = make_float4(h0, h1, h2, 0.0f);
        lo[i] = make_float4(l0, l1, l2, 0.0f);
    }
}

// double-float centres and weights: (c_hi, c_lo, w_hi, w_lo) per centre
__global__ void k_pack_centres_ff(const double *__restrict__ xb, const int32_t *__restrict__ sel,
                                  const double *__restrict__ w, int64_t nc, double inv_r,
                                  const unsigned long long *__restrict__ gmax,
                                  float4 *__restrict__ cff)
{
    const double G = grid_of(gmax);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nc;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = sel[j];
        float h0, l0, h1, l1, h2, l2;
        split_grid(xb[3 * n] * inv_r, G, h0, l0);
        split_grid(xb[3 * n + 1] * inv_r, G, h1, l1);
        split_grid(xb[3 * n + 2] * inv_r, G, h2, l2);
        cff[4 * j] = make_float4(h0, h1, h2, 0.0f);
        cff[4 * j + 1] = make_float4(l0, l1, l2, 0.0f);
        split_f64(w[3 * j], h0, l0);
        split_f64(w[3 * j + 1], h1, l1);
        split_f64(w[3 * j + 2], h2, l2);
        cff[4 * j + 2] = make_float4(h0, h1, h2, 0.0f);
        cff[4 * j + 3] = make_float4(l0, l1, l2, 0.0f);
    }
}

__global__ void k_fill_zero(double *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = 0.0;
}

// centres c_j = xb[sel[j]] / R and weights w_j, interleaved (c_j, w_j).
__global__ void k_pack_centres(const double *__restrict__ xb, const int32_t *__restrict__ sel,
                               const double *__restrict__ w, int64_t nc, double inv_r,
                               float4 *__restrict__ c32, D4 *__restrict__ c64)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nc;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = sel[j];
        const double cx = xb[3 * n] * inv_r, cy = xb[3 * n + 1] * inv_r, cz = xb[3 * n + 2] * inv_r;
        const double wx = w[3 * j], wy = w[3 * j + 1], wz = w[3 * j + 2];
        if (c32) {
            const float fx = (float)cx, fy = (float)cy, fz = (float)cz;
            const float gx = (float)wx, gy = (float)wy, gz = (float)wz;
            c32[3 * j] = make_float4(fx, fx, fy, fy);
            c32[3 * j + 1] = make_float4(fz, fz, gx, gx);
            c32[3 * j + 2] = make_float4(gy, gy, gz, gz);
        }
        if (c64) {
            c64[2 * j] = mk4(cx, cy, cz, 0.0);
            c64[2 * j + 1] = mk4(wx, wy, wz, 0.0);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 pair sum.  Each thread owns 2 * P volume points as P pairs in paired
// FP32 registers; the shared-memory table stores every centre duplicated,
// (cx, cx, cy, cy), (cz, cz, wx, wx), (wy, wy, wz, wz), so three broadcast
// 16-byte loads give the paired operands directly.  A pair of pairs costs 14
// paired instructions, two min and two MUFU square roots.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kVolThreads)
k_volume_f32(const float4 *__restrict__ xq, int64_t nv, const float4 *__restrict__ cw, int nc,
             double *__restrict__ out)
{
    extern __shared__ float4 s_cw[];
    const int tid = threadIdx.x;
    const int64_t per_block = (int64_t)kVolThreads * 2 * P;
    const bool one_tile = nc <= kTileF32;
    if (one_tile) {
        for (int j = tid; j < 3 * nc; j += kVolThreads)
            s_cw[j] = cw[j];
        __syncthreads();
    }
    for (int64_t base = blockIdx.x * per_block; base < nv; base += (int64_t)gridDim.x * per_block) {
        f2 qx[P], qy[P], qz[P], ax[P], ay[P], az[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int64_t v0 = base + (int64_t)(2 * i) * kVolThreads + tid;
            int64_t v1 = v0 + kVolThreads;
            v0 = v0 < nv ? v0 : nv - 1;
            v1 = v1 < nv ? v1 : nv - 1;
            const float4 p0 = xq[v0], p1 = xq[v1];
            qx[i] = f2_pack(p0.x, p1.x);
            qy[i] = f2_pack(p0.y, p1.y);
            qz[i] = f2_pack(p0.z, p1.z);
            ax[i] = f2_pack(0.0f, 0.0f);
            ay[i] = ax[i];
            az[i] = ax[i];
        }
        for (int t0 = 0; t0 < nc; t0 += kTileF32) {
            const int nt = min(kTileF32, nc - t0);
            if (!one_tile) {
                __syncthreads();
                for (int j = tid; j < 3 * nt; j += kVolThreads)
                    s_cw[j] = cw[3 * t0 + j];
                __syncthreads();
            }
#pragma unroll 2
            for (int j = 0; j < nt; ++j) {
                const float4 A = s_cw[3 * j], B = s_cw[3 * j + 1], C = s_cw[3 * j + 2];
                const f2 cx = f2_pack(A.x, A.y), cy = f2_pack(A.z, A.w), cz = f2_pack(B.x, B.y);
                const f2 wx = f2_pack(B.z, B.w), wy = f2_pack(C.x, C.y), wz = f2_pack(C.z, C.w);
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const f2 dx = f2_sub(qx[i], cx), dy = f2_sub(qy[i], cy), dz = f2_sub(qz[i], cz);
                    const f2 s = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                    const f2 ph = phi_f32x2_s(s);
                    ax[i] = f2_fma(wx, ph, ax[i]);
                    ay[i] = f2_fma(wy, ph, ay[i]);
                    az[i] = f2_fma(wz, ph, az[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float x0, x1, y0, y1, z0, z1;
            f2_unpack(ax[i], x0, x1);
            f2_unpack(ay[i], y0, y1);
            f2_unpack(az[i], z0, z1);
            const int64_t v0 = base + (int64_t)(2 * i) * kVolThreads + tid;
            const int64_t v1 = v0 + kVolThreads;
            if (v0 < nv) {
                out[3 * v0] = (double)x0;
                out[3 * v0 + 1] = (double)y0;
                out[3 * v0 + 2] = (double)z0;
            }
            if (v1 < nv) {
                out[3 * v1] = (double)x1;
                out[3 * v1 + 1] = (double)y1;
                out[3 * v1 + 2] = (double)z1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float pair sum: ~48-bit coordinates and weights, ~44-bit phi, ff
// accumulation; result h + l rounded to FP64.
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(kVolThreads)
k_volume_ff(const float4 *__restrict__ xh, const float4 *__restrict__ xl, int64_t nv,
            const float4 *__restrict__ cw, int nc, double *__restrict__ out)
{
    // Q points per thread, handled two at a time in paired registers
    static_assert(Q % 2 == 0, "points per thread come in pairs");
    constexpr int P = Q / 2;
    extern __shared__ float4 s_cwff[];
    const int tid = threadIdx.x;
    const int64_t per_block = (int64_t)kVolThreads * Q;
    const bool one_tile = nc <= kTileFF;
    if (one_tile) {
        for (int j = tid; j < 4 * nc; j += kVolThreads)
            s_cwff[j] = cw[j];
        __syncthreads();
    }
    for (int64_t base = blockIdx.x * per_block; base < nv; base += (int64_t)gridDim.x * per_block) {
        f2 qxh[P], qxl[P], qyh[P], qyl[P], qzh[P], qzl[P];
        ff2 ax[P], ay[P], az[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int64_t v0 = base + (int64_t)(2 * i) * kVolThreads + tid;
            int64_t v1 = v0 + kVolThreads;
            v0 = v0 < nv ? v0 : nv - 1;
            v1 = v1 < nv ? v1 : nv - 1;
            const float4 h0 = xh[v0], h1 = xh[v1], l0 = xl[v0], l1 = xl[v1];
            qxh[i] = f2_pack(h0.x, h1.x);
            qyh[i] = f2_pack(h0.y, h1.y);
            qzh[i] = f2_pack(h0.z, h1.z);
            qxl[i] = f2_pack(l0.x, l1.x);
            qyl[i] = f2_pack(l0.y, l1.y);
            qzl[i] = f2_pack(l0.z, l1.z);
            const f2 z = f2_pack(0.0f, 0.0f);
            ax[i] = ff2{z, z};
            ay[i] = ax[i];
            az[i] = ax[i];
        }
        for (int t0 = 0; t0 < nc; t0 += kTileFF) {
            const int nt = min(kTileFF, nc - t0);
            if (!one_tile) {
                __syncthreads();
                for (int j = tid; j < 4 * nt; j += kVolThreads)
                    s_cwff[j] = cw[4 * t0 + j];
                __syncthreads();
            }
            for (int j = 0; j < nt; ++j) {
                const float4 ch = s_cwff[4 * j], cl = s_cwff[4 * j + 1];
                const float4 wh = s_cwff[4 * j + 2], wl = s_cwff[4 * j + 3];
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const ff2 s2 = dist2_gs2(qxh[i], qxl[i], qyh[i], qyl[i], qzh[i], qzl[i],
                                             f2_bcast(ch.x), f2_bcast(cl.x), f2_bcast(ch.y),
                                             f2_bcast(cl.y), f2_bcast(ch.z), f2_bcast(cl.z));
                    const ff2 ph = phi_ff2_s(s2);
                    ff_fma_acc2(ax[i], f2_bcast(wh.x), f2_bcast(wl.x), ph);
                    ff_fma_acc2(ay[i], f2_bcast(wh.y), f2_bcast(wl.y), ph);
                    ff_fma_acc2(az[i], f2_bcast(wh.z), f2_bcast(wl.z), ph);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float xh0, xh1, xl0, xl1, yh0, yh1, yl0, yl1, zh0, zh1, zl0, zl1;
            f2_unpack(ax[i].h, xh0, xh1);
            f2_unpack(ax[i].l, xl0, xl1);
            f2_unpack(ay[i].h, yh0, yh1);
            f2_unpack(ay[i].l, yl0, yl1);
            f2_unpack(az[i].h, zh0, zh1);
            f2_unpack(az[i].l, zl0, zl1);
            const int64_t v0 = base + (int64_t)(2 * i) * kVolThreads + tid;
            const int64_t v1 = v0 + kVolThreads;
            if (v0 < nv) {
                out[3 * v0] = (double)xh0 + (double)xl0;
                out[3 * v0 + 1] = (double)yh0 + (double)yl0;
                out[3 * v0 + 2] = (double)zh0 + (double)zl0;
            }
            if (v1 < nv) {
                out[3 * v1] = (double)xh1 + (double)xl1;
                out[3 * v1 + 1] = (double)yh1 + (double)yl1;
                out[3 * v1 + 2] = (double)zh1 + (double)zl1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 pair sum (one point per thread).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVolThreads)
k_volume_f64(const double *__restrict__ xv, int64_t nv, double inv_r,
             const D4 *__restrict__ cw, int nc, double *__restrict__ out)
{
    extern __shared__ D4 s_cw64[];
    const int tid = threadIdx.x;
    for (int64_t base = blockIdx.x * (int64_t)kVolThreads; base < nv;
         base += (int64_t)gridDim.x * kVolThreads) {
        int64_t v = base + tid;
        const int64_t vc = v < nv ? v : nv - 1;
        const double qx = xv[3 * vc] * inv_r, qy = xv[3 * vc + 1] * inv_r, qz = xv[3 * vc + 2] * inv_r;
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int t0 = 0; t0 < nc; t0 += kTileF64) {
            const int nt = min(kTileF64, nc - t0);
            __syncthreads();
            for (int j = tid; j < 2 * nt; j += kVolThreads)
                s_cw64[j] = cw[2 * t0 + j];
            __syncthreads();
            for (int j = 0; j < nt; ++j) {
                const D4 c = s_cw64[2 * j];
                const D4 w = s_cw64[2 * j + 1];
                const double dx = qx - c.x, dy = qy - c.y, dz = qz - c.z;
                const double s = fma(dz, dz, fma(dy, dy, dx * dx));
                const double ph = phi_f64_s(s);
                ax = fma(w.x, ph, ax);
                ay = fma(w.y, ph, ay);
                az = fma(w.z, ph, az);
            }
        }
        if (v < nv) {
            out[3 * v] = ax;
            out[3 * v + 1] = ay;
            out[3 * v + 2] = az;
        }
    }
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
struct VolumeWs {
    size_t off_gmax, off_xq32, off_c32, off_c64, off_xh, off_xl, off_cff, total;
};

static VolumeWs volume_ws_layout(int64_t nv, int64_t nc, int prec)
{
    VolumeWs L{};
    size_t o = 0;
    L.off_gmax = o;
    o = 256;
    L.off_xq32 = o;
    if (prec == RBF_PREC_F32)
        o = align_up(o + sizeof(float4) * (size_t)nv, 256);
    L.off_c32 = o;
    if (prec == RBF_PREC_F32)
        o = align_up(o + sizeof(float4) * 3 * (size_t)nc, 256);
    L.off_c64 = o;
    if (prec == RBF_PREC_F64)
        o = align_up(o + sizeof(D4) * 2 * (size_t)nc, 256);
    L.off_xh = o;
    if (prec == RBF_PREC_F32X2)
        o = align_up(o + sizeof(float4) * (size_t)nv, 256);
    L.off_xl = o;
    if (prec == RBF_PREC_F32X2)
        o = align_up(o + sizeof(float4) * (size_t)nv, 256);
    L.off_cff = o;
    if (prec == RBF_PREC_F32X2)
        o = align_up(o + sizeof(float4) * 4 * (size_t)nc, 256);
    L.total = std::max<size_t>(o, 256);
    return L;
}

}  // namespace rbf

using namespace rbf;

extern "C" size_t rbf_volume_workspace_bytes(int64_t nv, int64_t nc, const rbf_params *p)
{
    if (!p || nv < 0 || nc < 0)
        return 0;
    return volume_ws_layout(nv, nc, p->eval_prec).total;
}

extern "C" rbf_status rbf_deform_volume(const double *d_xv, int64_t nv, const double *d_xb,
                                        const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                                        const rbf_params *p, double *d_dv, void *d_ws,
                                        size_t ws_bytes, void *stream)
{
    if (!p || nv < 0 || nc < 0 || !(p->radius > 0.0) ||
        (p->eval_prec != RBF_PREC_F32 && p->eval_prec != RBF_PREC_F64 &&
         p->eval_prec != RBF_PREC_F32X2))
        return RBF_E_ARG;
    if (nv == 0)
        return RBF_OK;
    if (!d_xv || !d_dv)
        return RBF_E_ARG;
    // the points and displacements may be pinned host memory the device can
    // reach (read and written once per point by the kernels)
    if (!device_accessible(d_xv) || !device_accessible(d_dv))
        return RBF_E_ARG;
    if (nc > 0 && (!d_xb || !d_sel_idx || !d_w))
        return RBF_E_ARG;
    if (nc > (int64_t)1 << 30 || nv > (int64_t)1 << 40)
        return RBF_E_ARG;
    const VolumeWs L = volume_ws_layout(nv, nc, p->eval_prec);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    const double inv_r = 1.0 / p->radius;
    if (nc == 0) {
        k_fill_zero<<<(int)std::min<int64_t>((3 * nv + 255) / 256, (int64_t)dev.sms * 8), 256, 0,
                      st>>>(d_dv, 3 * nv);
        return cudaGetLastError() == cudaSuccess ? RBF_OK : RBF_E_CUDA;
    }
    if (p->eval_prec == RBF_PREC_F32) {
        float4 *xq = (float4 *)(ws + L.off_xq32);
        float4 *c32 = (float4 *)(ws + L.off_c32);
        const int pb = (int)std::min<int64_t>((nv + 255) / 256, (int64_t)dev.sms * 8);
        k_pack_points_f32<<<pb, 256, 0, st>>>(d_xv, nv, inv_r, xq);
        const int cb = (int)std::min<int64_t>((nc + 255) / 256, (int64_t)dev.sms * 4);
        k_pack_centres<<<cb, 256, 0, st>>>(d_xb, d_sel_idx, d_w, nc, inv_r, c32, nullptr);
        const size_t smem = sizeof(float4) * 3 * (size_t)std::min<int64_t>(nc, kTileF32);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_volume_f32<kVolP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float4) * 3 * kTileF32));
            attr = true;
        }
        // resident CTAs per SM for this launch's shared-memory size
        int occ = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_volume_f32<kVolP>, kVolThreads,
                                                          smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
        const int64_t per = (int64_t)kVolThreads * 2 * kVolP;
        const int64_t want = (nv + per - 1) / per;
        const int grid = (int)std::min<int64_t>(want, (int64_t)dev.sms * occ);
        k_volume_f32<kVolP><<<grid, kVolThreads, smem, st>>>(xq, nv, c32, (int)nc, d_dv);
    } else if (p->eval_prec == RBF_PREC_F32X2) {
        float4 *xh = (float4 *)(ws + L.off_xh), *xl = (float4 *)(ws + L.off_xl);
        float4 *cff = (float4 *)(ws + L.off_cff);
        unsigned long long *gmax = (unsigned long long *)(ws + L.off_gmax);
        const int pb = (int)std::min<int64_t>((nv + 255) / 256, (int64_t)dev.sms * 8);
        if (cudaMemsetAsync(gmax, 0, sizeof(*gmax), st) != cudaSuccess)
            return RBF_E_CUDA;
        k_grid_max<<<pb, 256, 0, st>>>(d_xv, nv, d_xb, d_sel_idx, nc, inv_r, gmax);
        k_pack_points_ff<<<pb, 256, 0, st>>>(d_xv, nv, inv_r, gmax, xh, xl);
        const int cb = (int)std::min<int64_t>((nc + 255) / 256, (int64_t)dev.sms * 4);
        k_pack_centres_ff<<<cb, 256, 0, st>>>(d_xb, d_sel_idx, d_w, nc, inv_r, gmax, cff);
        const size_t smem = sizeof(float4) * 4 * (size_t)std::min<int64_t>(nc, kTileFF);
        static bool attr_ff = false;
        if (!attr_ff) {
            cudaFuncSetAttribute(k_volume_ff<kVolQFF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float4) * 4 * kTileFF));
            attr_ff = true;
        }
        int occ_ff = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ff, k_volume_ff<kVolQFF>, kVolThreads,
                                                          smem) != cudaSuccess ||
            occ_ff < 1)
            occ_ff = 1;
        const int64_t want =
            (nv + (int64_t)kVolThreads * kVolQFF - 1) / ((int64_t)kVolThreads * kVolQFF);
        const int grid = (int)std::min<int64_t>(want, (int64_t)dev.sms * occ_ff);
        k_volume_ff<kVolQFF><<<grid, kVolThreads, smem, st>>>(xh, xl, nv, cff, (int)nc, d_dv);
    } else {
        D4 *c64 = (D4 *)(ws + L.off_c64);
        const int cb = (int)std::min<int64_t>((nc + 255) / 256, (int64_t)dev.sms * 4);
        k_pack_centres<<<cb, 256, 0, st>>>(d_xb, d_sel_idx, d_w, nc, inv_r, nullptr, c64);
        const size_t smem = sizeof(D4) * 2 * (size_t)std::min<int64_t>(nc, kTileF64);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_volume_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(D4) * 2 * kTileF64));
            attr = true;
        }
        const int64_t want = (nv + kVolThreads - 1) / kVolThreads;
        const int grid = (int)std::min<int64_t>(want, (int64_t)dev.sms * 8);
        k_volume_f64<<<grid, kVolThreads, smem, st>>>(d_xv, nv, inv_r, c64, (int)nc, d_dv);
    }
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    return RBF_OK;
}

namespace rbf {

// ---------------------------------------------------------------------------
// Many displacement fields on one support set (Eq. 6 for every column of
// W, nc x n_out): D = Phi_vc W in double-float on the FP32 pipe.  Phi is
// computed once per (point, centre) pair into shared memory and shared by
// all n_out columns, so a pair costs one double-float phi plus n_out
// double-float multiply-adds instead of n_out / 3 separate volume sums.
//   CTA: 256 threads = PP point pairs x FG column groups of F columns (12
//   when n_out <= 96: two CTAs per SM; else 24);
//   a warp shares its column group (weights read as broadcasts) and covers
//   32 consecutive point pairs (phi entries read conflict-free).
//   Per centre tile of kFieldsK centres: stage the weights (w_hi, w_hi,
//   w_lo, w_lo per column, so one 16-byte load gives both paired operands),
//   compute the tile's phi (each thread kFieldsK / FG centres of its point
//   pair), then accumulate.  Accumulators are renormalised (error-free
//   two_sum) every kFieldsRenorm centres, which bounds the growth of their low
//   parts.
// ---------------------------------------------------------------------------
constexpr int kFieldsFMax = 24;       // columns per thread (12 or 24)
constexpr int kFieldsK = 32;          // centres per shared-memory tile
constexpr int kFieldsThreads = 256;
constexpr int kFieldsMaxOut = 192;    // 8 column groups
constexpr int kFieldsRenorm = 8;

static int fields_cols(int n_out) { return n_out <= 96 ? 12 : kFieldsFMax; }

static int fields_pad(int n_out)
{
    const int f = fields_cols(n_out);
    int np = f;
    while (np < n_out)
        np *= 2;
    return np;   // f, 2f, 4f or 8f: FG = np / f divides 8
}

__global__ void k_pack_fields_w(const double *__restrict__ w, int nc, int n_out, int n_pad,
                                float4 *__restrict__ wp)
{
    const int64_t tot = (int64_t)nc * n_pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / n_pad;
        const int f = (int)(i - j * n_pad);
        float h = 0.0f, l = 0.0f;
        if (f < n_out)
            split_f64(w[j * n_out + f], h, l);
        wp[i] = make_float4(h, h, l, l);
    }
}

// double-float centres: (c_hi, c_lo) per centre
__global__ void k_pack_centres_hl(const double *__restrict__ xb, const int32_t *__restrict__ sel,
                                  int64_t nc, double inv_r,
                                  const unsigned long long *__restrict__ gmax,
                                  float4 *__restrict__ c)
{
    const double G = grid_of(gmax);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nc;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = sel[j];
        float h0, l0, h1, l1, h2, l2;
        split_grid(xb[3 * n] * inv_r, G, h0, l0);
        split_grid(xb[3 * n + 1] * inv_r, G, h1, l1);
        split_grid(xb[3 * n + 2] * inv_r, G, h2, l2);
        c[2 * j] = make_float4(h0, h1, h2, 0.0f);
        c[2 * j + 1] = make_float4(l0, l1, l2, 0.0f);
    }
}

template <int FG, int F>
__global__ void __launch_bounds__(kFieldsThreads, F <= 12 ? 2 : 1)
k_fields_ff(const float4 *__restrict__ xh, const float4 *__restrict__ xl, int64_t nv,
            const float4 *__restrict__ c, int nc, const float4 *__restrict__ wp, int n_out,
            double *__restrict__ out)
{
    constexpr int PP = kFieldsThreads / FG;      // point pairs per CTA
    constexpr int NP = FG * F;                   // padded columns
    static_assert(PP % 32 == 0, "a warp must share one column group");
    extern __shared__ float4 s_f[];
    float4 *s_w = s_f;                           // [kFieldsK][NP]
    float4 *s_phi = s_f + kFieldsK * NP;         // [kFieldsK][PP]: (h0, h1, l0, l1)
    const int tid = threadIdx.x;
    const int pp = tid % PP, fg = tid / PP;
    const int64_t per_block = 2 * (int64_t)PP;
    for (int64_t base = blockIdx.x * per_block; base < nv; base += (int64_t)gridDim.x * per_block) {
        int64_t v0 = base + pp, v1 = base + PP + pp;
        const int64_t r0 = v0 < nv ? v0 : nv - 1, r1 = v1 < nv ? v1 : nv - 1;
        const float4 h0 = xh[r0], h1 = xh[r1], l0 = xl[r0], l1 = xl[r1];
        const f2 qxh = f2_pack(h0.x, h1.x), qyh = f2_pack(h0.y, h1.y), qzh = f2_pack(h0.z, h1.z);
        const f2 qxl = f2_pack(l0.x, l1.x), qyl = f2_pack(l0.y, l1.y), qzl = f2_pack(l0.z, l1.z);
        const f2 z = f2_pack(0.0f, 0.0f);
        ff2 acc[F];
#pragma unroll
        for (int f = 0; f < F; ++f)
            acc[f] = ff2{z, z};
        int nren = 0;
        for (int t0 = 0; t0 < nc; t0 += kFieldsK) {
            const int nt = min(kFieldsK, nc - t0);
            __syncthreads();   // the previous tile's readers are done
            for (int i = tid; i < nt * NP; i += kFieldsThreads)
                s_w[i] = wp[(int64_t)t0 * NP + i];
            for (int k = fg; k < nt; k += FG) {
                const float4 ch = __ldg(c + 2 * (t0 + k)), cl = __ldg(c + 2 * (t0 + k) + 1);
                const ff2 s2 = dist2_gs2(qxh, qxl, qyh, qyl, qzh, qzl, f2_bcast(ch.x),
                                         f2_bcast(cl.x), f2_bcast(ch.y), f2_bcast(cl.y),
                                         f2_bcast(ch.z), f2_bcast(cl.z));
                const ff2 ph = phi_ff2_s(s2);
                float a0, a1, b0, b1;
                f2_unpack(ph.h, a0, a1);
                f2_unpack(ph.l, b0, b1);
                s_phi[k * PP + pp] = make_float4(a0, a1, b0, b1);
            }
            __syncthreads();
            for (int k = 0; k < nt; ++k) {
                if (++nren == kFieldsRenorm) {
                    nren = 0;
#pragma unroll
                    for (int f = 0; f < F; ++f)
                        acc[f] = two_sum2(acc[f].h, acc[f].l);
                }
                const float4 pv = s_phi[k * PP + pp];
                const ff2 ph{f2_pack(pv.x, pv.y), f2_pack(pv.z, pv.w)};
                const float4 *wk = s_w + k * NP + fg * F;
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    const float4 w = wk[f];
                    ff_fma_acc2(acc[f], f2_pack(w.x, w.y), f2_pack(w.z, w.w), ph);
                }
            }
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int col = fg * F + f;
            if (col < n_out) {
                float hh0, hh1, ll0, ll1;
                f2_unpack(acc[f].h, hh0, hh1);
                f2_unpack(acc[f].l, ll0, ll1);
                if (v0 < nv)
                    out[v0 * n_out + col] = (double)hh0 + (double)ll0;
                if (v1 < nv)
                    out[v1 * n_out + col] = (double)hh1 + (double)ll1;
            }
        }
    }
}

struct FieldsWs {
    size_t gmax, xh, xl, c, w, total;
};

static FieldsWs fields_ws(int64_t nv, int64_t nc, int n_out)
{
    FieldsWs L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.gmax = take(sizeof(unsigned long long));
    L.xh = take(sizeof(float4) * (size_t)nv);
    L.xl = take(sizeof(float4) * (size_t)nv);
    L.c = take(sizeof(float4) * 2 * (size_t)std::max<int64_t>(nc, 1));
    L.w = take(sizeof(float4) * (size_t)std::max<int64_t>(nc, 1) * fields_pad(n_out));
    L.total = o;
    return L;
}

}  // namespace rbf

extern "C" size_t rbf_volume_fields_workspace_bytes(int64_t nv, int64_t nc, int n_out)
{
    using namespace rbf;
    if (nv < 0 || nc < 0 || n_out < 1 || n_out > kFieldsMaxOut)
        return 0;
    return fields_ws(nv, nc, n_out).total;
}

extern "C" rbf_status rbf_deform_volume_fields(const double *d_xv, int64_t nv, const double *d_xb,
                                               const int32_t *d_sel_idx, int64_t nc,
                                               const double *d_w, int n_out, const rbf_params *p,
                                               double *d_out, void *d_ws, size_t ws_bytes,
                                               void *stream)
{
    using namespace rbf;
    if (!p || !(p->radius > 0.0) || !std::isfinite(p->radius) || p->eval_prec != RBF_PREC_F32X2 ||
        nv < 0 || nc < 0 || nc > INT32_MAX / kFieldsMaxOut || n_out < 1 || n_out > kFieldsMaxOut)
        return RBF_E_ARG;
    if (nv == 0)
        return RBF_OK;
    if (!d_xv || !d_out || (nc > 0 && (!d_xb || !d_sel_idx || !d_w)))
        return RBF_E_ARG;
    const FieldsWs L = fields_ws(nv, nc, n_out);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (nc == 0) {
        if (cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)nv * n_out, st) != cudaSuccess)
            return RBF_E_CUDA;
        return RBF_OK;
    }
    char *ws = (char *)d_ws;
    float4 *xh = (float4 *)(ws + L.xh), *xl = (float4 *)(ws + L.xl);
    float4 *c = (float4 *)(ws + L.c), *wp = (float4 *)(ws + L.w);
    const double inv_r = 1.0 / p->radius;
    const int n_pad = fields_pad(n_out);
    const int fcols = fields_cols(n_out);
    const int fg = n_pad / fcols;
    unsigned long long *gmax = (unsigned long long *)(ws + L.gmax);
    const int pb = (int)std::min<int64_t>((nv + 255) / 256, (int64_t)dev.sms * 8);
    if (cudaMemsetAsync(gmax, 0, sizeof(*gmax), st) != cudaSuccess)
        return RBF_E_CUDA;
    k_grid_max<<<pb, 256, 0, st>>>(d_xv, nv, d_xb, d_sel_idx, nc, inv_r, gmax);
    k_pack_points_ff<<<pb, 256, 0, st>>>(d_xv, nv, inv_r, gmax, xh, xl);
    k_pack_centres_hl<<<(int)std::min<int64_t>((nc + 255) / 256, (int64_t)dev.sms * 4), 256, 0,
                        st>>>(d_xb, d_sel_idx, nc, inv_r, gmax, c);
    const int64_t wtot = nc * n_pad;
    k_pack_fields_w<<<(int)std::min<int64_t>((wtot + 255) / 256, (int64_t)dev.sms * 8), 256, 0,
                      st>>>(d_w, (int)nc, n_out, n_pad, wp);
    const int pp = kFieldsThreads / fg;
    const size_t smem = sizeof(float4) * (size_t)kFieldsK * (n_pad + pp);
    const int64_t tiles = (nv + 2 * pp - 1) / (2 * pp);
#define RBF_FIELDS_LAUNCH(FGV, FV)                                                            \
    do {                                                                                      \
        if (cudaFuncSetAttribute(k_fields_ff<FGV, FV>,                                        \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=   \
            cudaSuccess)                                                                      \
            return RBF_E_CUDA;                                                                \
        int occ = 1;                                                                          \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fields_ff<FGV, FV>,         \
                                                          kFieldsThreads, smem) != cudaSuccess || \
            occ < 1)                                                                          \
            occ = 1;                                                                          \
        const int grid = (int)std::min<int64_t>(tiles, (int64_t)dev.sms * occ);               \
        k_fields_ff<FGV, FV><<<grid, kFieldsThreads, smem, st>>>(xh, xl, nv, c, (int)nc, wp,  \
                                                                 n_out, d_out);               \
    } while (0)
    if (fcols == 12) {
        if (fg == 1)
            RBF_FIELDS_LAUNCH(1, 12);
        else if (fg == 2)
            RBF_FIELDS_LAUNCH(2, 12);
        else if (fg == 4)
            RBF_FIELDS_LAUNCH(4, 12);
        else
            RBF_FIELDS_LAUNCH(8, 12);
    } else {
        RBF_FIELDS_LAUNCH(8, 24);
    }
#undef RBF_FIELDS_LAUNCH
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    return RBF_OK;
}

// ---------------------------------------------------------------------------
// Batched volume sums: many problems (each its own points, support set and
// weights) in one launch of the double-float kernel.  Work items are tiles of
// THREADS * P points; CTA b takes a contiguous run of items, so it reloads
// the shared-memory centre table only when its run crosses into the next
// problem.  The tile shape is chosen at create time by timing the candidate
// instantiations on the real problems (self-written autotuner).
// ---------------------------------------------------------------------------
namespace rbf {

struct VolProbDev {
    const double *xv;
    int64_t nv;
    const float4 *table;      // (c_hi, c_lo, w_hi, w_lo) per centre
    const int64_t *nc;        // device count of centres
    double *dv;
    double inv_r;
    int64_t item0;            // first work item of the problem
};

__global__ void k_vb_pack(const rbf_volume_problem *__restrict__ probs, int B,
                          float4 *const *__restrict__ tables, int max_nc)
{
    const int i = blockIdx.y;
    if (i >= B)
        return;
    const rbf_volume_problem q = probs[i];
    const int nc = (int)min((int64_t)max_nc, *q.d_nc);
    const double inv_r = 1.0 / q.radius;
    float4 *t = tables[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        const int64_t n = q.d_sel_idx[j];
        float h0, l0, h1, l1, h2, l2;
        split_f64(q.d_xb[3 * n] * inv_r, h0, l0);
        split_f64(q.d_xb[3 * n + 1] * inv_r, h1, l1);
        split_f64(q.d_xb[3 * n + 2] * inv_r, h2, l2);
        t[4 * j] = make_float4(h0, h1, h2, 0.0f);
        t[4 * j + 1] = make_float4(l0, l1, l2, 0.0f);
        split_f64(q.d_w[3 * j], h0, l0);
        split_f64(q.d_w[3 * j + 1], h1, l1);
        split_f64(q.d_w[3 * j + 2], h2, l2);
        t[4 * j + 2] = make_float4(h0, h1, h2, 0.0f);
        t[4 * j + 3] = make_float4(l0, l1, l2, 0.0f);
    }
}

template <int THREADS, int P>
__global__ void __launch_bounds__(THREADS)
k_vb_volume_ff(const VolProbDev *__restrict__ probs, int B, int64_t n_items, int64_t per_cta)
{
    extern __shared__ float4 s_tab[];
    const int tid = threadIdx.x;
    const int64_t it0 = (int64_t)blockIdx.x * per_cta;
    const int64_t it1 = min(n_items, it0 + per_cta);
    int cur = -1, nc = 0;
    VolProbDev q{};
    for (int64_t it = it0; it < it1; ++it) {
        // problem of this item: last i with item0 <= it
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (probs[mid].item0 <= it)
                lo = mid;
            else
                hi = mid - 1;
        }
        if (lo != cur) {
            cur = lo;
            q = probs[cur];
            nc = (int)*q.nc;
            __syncthreads();
            for (int j = tid; j < 4 * nc; j += THREADS)
                s_tab[j] = q.table[j];
            __syncthreads();
        }
        const int64_t base = (it - q.item0) * (int64_t)THREADS * P;
        float qh[P][3], ql[P][3];
        ff acc[P][3];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int64_t v = base + (int64_t)i * THREADS + tid;
            v = v < q.nv ? v : q.nv - 1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                split_f64(q.xv[3 * v + c] * q.inv_r, qh[i][c], ql[i][c]);
                acc[i][c] = ff{0.0f, 0.0f};
            }
        }
        for (int j = 0; j < nc; ++j) {
            const float4 ch = s_tab[4 * j], cl = s_tab[4 * j + 1];
            const float4 wh = s_tab[4 * j + 2], wl = s_tab[4 * j + 3];
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const ff s2 = dist2_ff(qh[i][0], ql[i][0], qh[i][1], ql[i][1], qh[i][2], ql[i][2],
                                       ch.x, cl.x, ch.y, cl.y, ch.z, cl.z);
                const ff ph = phi_ff_s(s2);
                ff_fma_acc(acc[i][0], wh.x, wl.x, ph);
                ff_fma_acc(acc[i][1], wh.y, wl.y, ph);
                ff_fma_acc(acc[i][2], wh.z, wl.z, ph);
            }
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int64_t v = base + (int64_t)i * THREADS + tid;
            if (v < q.nv)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    q.dv[3 * v + c] = (double)acc[i][c].h + (double)acc[i][c].l;
        }
    }
}

constexpr int kVbMaxCentres = 1024;   // shared-memory table: 64 KB

struct VbCandidate {
    int threads, p;
};
static const VbCandidate kVbCands[4] = {{128, 1}, {128, 2}, {256, 1}, {256, 2}};

struct VbLayout {
    size_t probs_host, probs_dev, tables_ptr, tables, total;
};

static VbLayout vb_layout(int B, int64_t sum_ncmax)
{
    VbLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.probs_host = take(sizeof(rbf_volume_problem) * (size_t)B);
    L.probs_dev = take(sizeof(VolProbDev) * (size_t)B);
    L.tables_ptr = take(sizeof(float4 *) * (size_t)B);
    L.tables = take(sizeof(float4) * 4 * (size_t)sum_ncmax);
    L.total = o;
    return L;
}

}  // namespace rbf

struct rbf_volume_batch {
    int B = 0;
    int cand = 0;
    int grid = 0;
    int64_t n_items = 0, per_cta = 0;
    int max_nc = 0;
    char *ws = nullptr;
    size_t probs_host = 0, probs_dev = 0, tables_ptr = 0;
    float cand_ms[4] = {0, 0, 0, 0};
};

namespace rbf {
static cudaError_t vb_launch(const rbf_volume_batch *b, int cand, cudaStream_t st)
{
    const rbf_volume_problem *ph = (const rbf_volume_problem *)(b->ws + b->probs_host);
    float4 *const *tp = (float4 *const *)(b->ws + b->tables_ptr);
    k_vb_pack<<<dim3(4, b->B), 256, 0, st>>>(ph, b->B, tp, b->max_nc);
    const VbCandidate c = kVbCands[cand];
    const int64_t tile = (int64_t)c.threads * c.p;
    (void)tile;
    const VolProbDev *pd = (const VolProbDev *)(b->ws + b->probs_dev);
    const size_t smem = sizeof(float4) * 4 * (size_t)b->max_nc;
    switch (cand) {
    case 0: k_vb_volume_ff<128, 1><<<b->grid, 128, smem, st>>>(pd, b->B, b->n_items, b->per_cta); break;
    case 1: k_vb_volume_ff<128, 2><<<b->grid, 128, smem, st>>>(pd, b->B, b->n_items, b->per_cta); break;
    case 2: k_vb_volume_ff<256, 1><<<b->grid, 256, smem, st>>>(pd, b->B, b->n_items, b->per_cta); break;
    default: k_vb_volume_ff<256, 2><<<b->grid, 256, smem, st>>>(pd, b->B, b->n_items, b->per_cta); break;
    }
    return cudaGetLastError();
}

// item layout depends on the tile size of the candidate
static rbf_status vb_configure(rbf_volume_batch *b, const rbf_volume_problem *h, int cand,
                               const std::vector<float4 *> &tables, cudaStream_t st, int sms)
{
    const VbCandidate c = kVbCands[cand];
    const int64_t tile = (int64_t)c.threads * c.p;
    std::vector<VolProbDev> pd(b->B);
    int64_t items = 0;
    for (int i = 0; i < b->B; ++i) {
        pd[i].xv = h[i].d_xv;
        pd[i].nv = h[i].nv;
        pd[i].table = tables[i];
        pd[i].nc = h[i].d_nc;
        pd[i].dv = h[i].d_dv;
        pd[i].inv_r = 1.0 / h[i].radius;
        pd[i].item0 = items;
        items += (h[i].nv + tile - 1) / tile;
    }
    b->n_items = items;
    b->grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * 8));
    b->per_cta = (items + b->grid - 1) / b->grid;
    b->grid = (int)((items + b->per_cta - 1) / b->per_cta);
    if (cudaMemcpyAsync(b->ws + b->probs_dev, pd.data(), sizeof(VolProbDev) * b->B,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RBF_E_CUDA;
    b->cand = cand;
    return RBF_OK;
}
}  // namespace rbf

extern "C" size_t rbf_volume_batch_workspace_bytes(const rbf_volume_problem *h_probs, int B,
                                                   int eval_prec)
{
    if (!h_probs || B < 1 || eval_prec != RBF_PREC_F32X2)
        return 0;
    int64_t s = 0;
    for (int i = 0; i < B; ++i) {
        if (h_probs[i].nc_max < 1 || h_probs[i].nc_max > kVbMaxCentres)
            return 0;
        s += h_probs[i].nc_max;
    }
    return vb_layout(B, s).total;
}

extern "C" rbf_status rbf_volume_batch_create(const rbf_volume_problem *h_probs, int B,
                                              int eval_prec, void *d_ws, size_t ws_bytes,
                                              void *stream, rbf_volume_batch **out)
{
    if (!h_probs || B < 1 || !out || eval_prec != RBF_PREC_F32X2)
        return RBF_E_ARG;
    *out = nullptr;
    int64_t sum = 0;
    int max_nc = 0;
    for (int i = 0; i < B; ++i) {
        const rbf_volume_problem &q = h_probs[i];
        if (q.nv < 1 || q.nc_max < 1 || q.nc_max > kVbMaxCentres || !q.d_xv || !q.d_xb ||
            !q.d_sel_idx || !q.d_w || !q.d_nc || !q.d_dv || !(q.radius > 0.0))
            return RBF_E_ARG;
        sum += q.nc_max;
        max_nc = std::max<int>(max_nc, (int)q.nc_max);
    }
    const VbLayout L = vb_layout(B, sum);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    std::vector<float4 *> tables(B);
    size_t o = L.tables;
    for (int i = 0; i < B; ++i) {
        tables[i] = (float4 *)(ws + o);
        o += sizeof(float4) * 4 * (size_t)h_probs[i].nc_max;
    }
    if (cudaMemcpyAsync(ws + L.probs_host, h_probs, sizeof(rbf_volume_problem) * B,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.tables_ptr, tables.data(), sizeof(float4 *) * B,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RBF_E_CUDA;
    const size_t smem_max = sizeof(float4) * 4 * kVbMaxCentres;
    cudaFuncSetAttribute(k_vb_volume_ff<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    cudaFuncSetAttribute(k_vb_volume_ff<128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    cudaFuncSetAttribute(k_vb_volume_ff<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    cudaFuncSetAttribute(k_vb_volume_ff<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    rbf_volume_batch *b = new rbf_volume_batch();
    b->B = B;
    b->max_nc = max_nc;
    b->ws = ws;
    b->probs_host = L.probs_host;
    b->probs_dev = L.probs_dev;
    b->tables_ptr = L.tables_ptr;
    // autotune: time every candidate once (after one untimed run) on the
    // real problems and keep the fastest
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    for (int cnd = 0; cnd < 4; ++cnd) {
        if (vb_configure(b, h_probs, cnd, tables, st, dev.sms) != RBF_OK ||
            vb_launch(b, cnd, st) != cudaSuccess) {
            delete b;
            return RBF_E_CUDA;
        }
        cudaEventRecord(e0, st);
        vb_launch(b, cnd, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return RBF_E_CUDA;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->cand_ms[cnd] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = cnd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (vb_configure(b, h_probs, best, tables, st, dev.sms) != RBF_OK) {
        delete b;
        return RBF_E_CUDA;
    }
    *out = b;
    return RBF_OK;
}

extern "C" rbf_status rbf_volume_batch_run(rbf_volume_batch *b, void *stream)
{
    if (!b)
        return RBF_E_ARG;
    return vb_launch(b, b->cand, (cudaStream_t)stream) == cudaSuccess ? RBF_OK : RBF_E_CUDA;
}

extern "C" rbf_status rbf_volume_batch_info(const rbf_volume_batch *b, int *threads,
                                            int *points_per_thread, float *candidate_ms)
{
    if (!b)
        return RBF_E_ARG;
    if (threads)
        *threads = kVbCands[b->cand].threads;
    if (points_per_thread)
        *points_per_thread = kVbCands[b->cand].p;
    if (candidate_ms)
        for (int i = 0; i < 4; ++i)
            candidate_ms[i] = b->cand_ms[i];
    return RBF_OK;
}

extern "C" void rbf_volume_batch_destroy(rbf_volume_batch *b)
{
    delete b;
}
