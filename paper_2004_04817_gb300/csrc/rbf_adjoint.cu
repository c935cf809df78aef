// rbf_adjoint.cu -- adjoint of the volume deformation (Eq. 6 composed with
// the support solve of Eqs. 4-5) for shape-optimisation gradients:
//
//     d_v = Phi_vc W,  Phi_cc W = d_c   =>   dJ/dd_c = Phi_cc^-1 Phi_vc^T dJ/dd_v
//
// (Phi_cc is symmetric).  Phi is recomputed pair by pair, never stored.
//
// Stage 1 (k_adjoint_partial): every CTA owns a fixed set of volume-point
// chunks; a chunk of points (scaled coordinates and dJ/dd_v) is staged in
// shared memory and every thread accumulates, for its centres, the sum over
// the chunk of phi_vj g_v (FP32 or double-float pairs), then adds the chunk
// total to FP64 registers.  Stage 2 (k_adjoint_reduce) sums the per-CTA FP64
// partials of each centre in a fixed order (deterministic).  Stage 3 solves
// Phi_cc lambda = g_c in FP64 (rbf_solve_system).
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kAdjMaxCentres = 1024; // one centre per thread, one CTA of up to 1024
constexpr int kAdjChunk = 1024;      // volume points per shared-memory chunk

// Packing: scaled volume points and their gradients (hi/lo splits for the
// double-float path).
// Double-float path (gmax given): coordinates grid-split (split_grid) for
// exact pair differences; FP32 path: the FP32 rounding in the high part.
__device__ __forceinline__ void adj_split(double x, const unsigned long long *gmax, double G,
                                          float &h, float &l)
{
    if (gmax)
        split_grid(x, G, h, l);
    else
        split_f64(x, h, l);
}

__global__ void k_adjoint_pack(const double *__restrict__ xv, const double *__restrict__ gv,
                               int64_t nv, double inv_r, const unsigned long long *gmax,
                               float4 *__restrict__ xh, float4 *__restrict__ xl,
                               float4 *__restrict__ gh, float4 *__restrict__ gl)
{
    const double G = gmax ? grid_of(gmax) : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h0, l0, h1, l1, h2, l2;
        adj_split(xv[3 * i] * inv_r, gmax, G, h0, l0);
        adj_split(xv[3 * i + 1] * inv_r, gmax, G, h1, l1);
        adj_split(xv[3 * i + 2] * inv_r, gmax, G, h2, l2);
        xh[i] = make_float4(h0, h1, h2, 0.0f);
        xl[i] = make_float4(l0, l1, l2, 0.0f);
        split_f64(gv[3 * i], h0, l0);
        split_f64(gv[3 * i + 1], h1, l1);
        split_f64(gv[3 * i + 2], h2, l2);
        gh[i] = make_float4(h0, h1, h2, 0.0f);
        gl[i] = make_float4(l0, l1, l2, 0.0f);
    }
}

__global__ void k_adjoint_centres(const double *__restrict__ xb, const int32_t *__restrict__ sel,
                                  int nc, double inv_r, const unsigned long long *gmax,
                                  float4 *__restrict__ ch, float4 *__restrict__ cl)
{
    const double G = gmax ? grid_of(gmax) : 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        const int64_t n = sel[j];
        float h0, l0, h1, l1, h2, l2;
        adj_split(xb[3 * n] * inv_r, gmax, G, h0, l0);
        adj_split(xb[3 * n + 1] * inv_r, gmax, G, h1, l1);
        adj_split(xb[3 * n + 2] * inv_r, gmax, G, h2, l2);
        ch[j] = make_float4(h0, h1, h2, 0.0f);
        cl[j] = make_float4(l0, l1, l2, 0.0f);
    }
}

// One centre per thread: the CTA has nc threads rounded up to a warp (<= 1024),
// so every thread has the same work; each chunk of points is staged in
// shared memory and read by all threads as broadcasts.
template <bool FF>
__global__ void __launch_bounds__(1024)
k_adjoint_partial(const float4 *__restrict__ xh, const float4 *__restrict__ xl,
                  const float4 *__restrict__ gh, const float4 *__restrict__ gl, int64_t nv,
                  const float4 *__restrict__ ch, const float4 *__restrict__ cl, int nc,
                  double *__restrict__ partial)
{
    extern __shared__ float4 s_pts[];     // [chunk] x_hi, x_lo, g_hi, g_lo
    float4 *s_xh = s_pts, *s_xl = s_pts + kAdjChunk, *s_gh = s_pts + 2 * kAdjChunk,
           *s_gl = s_pts + 3 * kAdjChunk;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool mine = tid < nc;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    const float4 qh = mine ? ch[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 ql = mine ? cl[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t nchunks = (nv + kAdjChunk - 1) / kAdjChunk;
    for (int64_t ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
        const int64_t v0 = ck * kAdjChunk;
        const int nvc = (int)min((int64_t)kAdjChunk, nv - v0);
        __syncthreads();
        for (int i = tid; i < nvc; i += nthr) {
            s_xh[i] = xh[v0 + i];
            s_gh[i] = gh[v0 + i];
            if (FF) {
                s_xl[i] = xl[v0 + i];
                s_gl[i] = gl[v0 + i];
            }
        }
        __syncthreads();
        if (!mine)
            continue;
        if (!FF) {
            float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll 4
            for (int i = 0; i < nvc; ++i) {
                const float4 x = s_xh[i], g = s_gh[i];
                const float dx = x.x - qh.x, dy = x.y - qh.y, dz = x.z - qh.z;
                const float ph = phi_f32_s(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                ax = fmaf(g.x, ph, ax);
                ay = fmaf(g.y, ph, ay);
                az = fmaf(g.z, ph, az);
            }
            acc0 += (double)ax;
            acc1 += (double)ay;
            acc2 += (double)az;
        } else {
            ff ax{0.0f, 0.0f}, ay{0.0f, 0.0f}, az{0.0f, 0.0f};
#pragma unroll 2
            for (int i = 0; i < nvc; ++i) {
                const float4 x0 = s_xh[i], x1 = s_xl[i];
                const float4 g0 = s_gh[i], g1 = s_gl[i];
                const ff s2 = dist2_gs(x0.x, x1.x, x0.y, x1.y, x0.z, x1.z, qh.x, ql.x, qh.y,
                                       ql.y, qh.z, ql.z);
                const ff ph = phi_ff_s(s2);
                ff_fma_acc(ax, g0.x, g1.x, ph);
                ff_fma_acc(ay, g0.y, g1.y, ph);
                ff_fma_acc(az, g0.z, g1.z, ph);
            }
            acc0 += (double)ax.h + (double)ax.l;
            acc1 += (double)ay.h + (double)ay.l;
            acc2 += (double)az.h + (double)az.l;
        }
    }
    if (mine) {
        double *pp = partial + ((size_t)blockIdx.x * nc + tid) * 3;
        pp[0] = acc0;
        pp[1] = acc1;
        pp[2] = acc2;
    }
}

// g_c[j][k] = sum over CTAs b (in order) of partial[b][j][k].
__global__ void k_adjoint_reduce(const double *__restrict__ partial, int nblocks, int nc,
                                 double *__restrict__ gc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nc)
        return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b)
        s += partial[(size_t)b * 3 * nc + t];
    gc[t] = s;
}

struct AdjWs {
    size_t gmax, xh, xl, gh, gl, ch, cl, partial, gc, solve, total;
    int blocks;
};

static AdjWs adjoint_ws_layout(int64_t nv, int64_t nc, int blocks)
{
    AdjWs L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.gmax = take(sizeof(unsigned long long));
    L.xh = take(sizeof(float4) * nv);
    L.xl = take(sizeof(float4) * nv);
    L.gh = take(sizeof(float4) * nv);
    L.gl = take(sizeof(float4) * nv);
    L.ch = take(sizeof(float4) * nc);
    L.cl = take(sizeof(float4) * nc);
    L.partial = take(sizeof(double) * 3 * (size_t)nc * blocks);
    L.gc = take(sizeof(double) * 3 * nc);
    L.solve = take(rbf_solve_workspace_bytes(nc));
    L.total = o;
    L.blocks = blocks;
    return L;
}

static int adjoint_blocks()
{
    DeviceInfo dev;
    if (!device_info(&dev))
        return 152 * 8;
    return dev.sms * 8;
}

}  // namespace rbf

using namespace rbf;

extern "C" size_t rbf_adjoint_workspace_bytes(int64_t nv, int64_t nc)
{
    if (nv < 0 || nc < 1 || nc > kAdjMaxCentres)
        return 0;
    return adjoint_ws_layout(nv, nc, adjoint_blocks()).total;
}

// Stages 1-2: g_c = Phi_vc^T g_v into gc (workspace), ASYNC.
static rbf_status adjoint_rhs(const double *d_xv, int64_t nv, const double *d_xb,
                              const int32_t *d_sel_idx, int64_t nc, const double *d_gv,
                              double radius, int eval_prec, const AdjWs &L, char *ws,
                              cudaStream_t st)
{
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    const double inv_r = 1.0 / radius;
    float4 *xh = (float4 *)(ws + L.xh), *xl = (float4 *)(ws + L.xl);
    float4 *gh = (float4 *)(ws + L.gh), *gl = (float4 *)(ws + L.gl);
    float4 *ch = (float4 *)(ws + L.ch), *cl = (float4 *)(ws + L.cl);
    double *partial = (double *)(ws + L.partial), *gc = (double *)(ws + L.gc);
    const int blocks = (int)std::min<int64_t>(L.blocks, std::max<int64_t>(
                                                            (nv + kAdjChunk - 1) / kAdjChunk, 1));
    const bool ffm = eval_prec == RBF_PREC_F32X2;
    unsigned long long *gmax = ffm ? (unsigned long long *)(ws + L.gmax) : nullptr;
    const int pb = (int)std::min<int64_t>((std::max<int64_t>(nv, nc) + 255) / 256,
                                          (int64_t)dev.sms * 8);
    if (ffm) {
        if (cudaMemsetAsync(gmax, 0, sizeof(*gmax), st) != cudaSuccess)
            return RBF_E_CUDA;
        k_grid_max<<<pb, 256, 0, st>>>(d_xv, nv, d_xb, d_sel_idx, nc, inv_r, gmax);
    }
    if (nv > 0)
        k_adjoint_pack<<<pb, 256, 0, st>>>(d_xv, d_gv, nv, inv_r, gmax, xh, xl, gh, gl);
    k_adjoint_centres<<<(int)((nc + 127) / 128), 128, 0, st>>>(d_xb, d_sel_idx, (int)nc, inv_r,
                                                                gmax, ch, cl);
    const size_t smem = sizeof(float4) * 4 * kAdjChunk;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_adjoint_partial<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cudaFuncSetAttribute(k_adjoint_partial<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int threads = (int)((nc + 31) / 32 * 32);
    if (ffm)
        k_adjoint_partial<true><<<blocks, threads, smem, st>>>(xh, xl, gh, gl, nv, ch, cl,
                                                               (int)nc, partial);
    else
        k_adjoint_partial<false><<<blocks, threads, smem, st>>>(xh, xl, gh, gl, nv, ch, cl,
                                                                (int)nc, partial);
    k_adjoint_reduce<<<(int)((3 * nc + 127) / 128), 128, 0, st>>>(partial, blocks, (int)nc, gc);
    return cudaGetLastError() == cudaSuccess ? RBF_OK : RBF_E_CUDA;
}

extern "C" rbf_status rbf_deform_volume_adjoint(const double *d_xv, int64_t nv,
                                                const double *d_xb, int64_t nb,
                                                const int32_t *d_sel_idx, int64_t nc,
                                                const double *d_gv, const rbf_params *p,
                                                double *d_gc, double *h_max_resid, void *d_ws,
                                                size_t ws_bytes, void *stream)
{
    if (!p || nv < 0 || nc < 1 || nc > kAdjMaxCentres || nc > nb ||
        !(p->radius > 0.0) || !d_xb || !d_sel_idx || !d_gc ||
        (nv > 0 && (!d_xv || !d_gv)) ||
        (p->eval_prec != RBF_PREC_F32 && p->eval_prec != RBF_PREC_F32X2))
        return RBF_E_ARG;
    const AdjWs L = adjoint_ws_layout(nv, nc, adjoint_blocks());
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    char *ws = (char *)d_ws;
    const rbf_status s = adjoint_rhs(d_xv, nv, d_xb, d_sel_idx, nc, d_gv, p->radius,
                                     p->eval_prec, L, ws, (cudaStream_t)stream);
    if (s != RBF_OK)
        return s;
    // Phi_cc lambda = g_c (symmetric, FP64 factor + refinement)
    rbf_params ps = *p;
    return rbf_solve_system(d_xb, nb, d_sel_idx, nc, (const double *)(ws + L.gc), &ps, d_gc,
                            h_max_resid, ws + L.solve, ws_bytes - L.solve, stream);
}

extern "C" rbf_status rbf_deform_volume_adjoint_factored(const double *d_xv, int64_t nv,
                                                         const double *d_gv, const rbf_factor *f,
                                                         const rbf_params *p, double *d_gc,
                                                         double *h_max_resid, void *d_ws,
                                                         size_t ws_bytes, void *stream)
{
    if (!p || !f || nv < 0 || f->nc > kAdjMaxCentres || !d_gc ||
        (nv > 0 && (!d_xv || !d_gv)) || p->refine_steps < 0 || p->refine_steps > 15 ||
        (p->eval_prec != RBF_PREC_F32 && p->eval_prec != RBF_PREC_F32X2))
        return RBF_E_ARG;
    const AdjWs L = adjoint_ws_layout(nv, f->nc, adjoint_blocks());
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    char *ws = (char *)d_ws;
    const rbf_status s = adjoint_rhs(d_xv, nv, f->xb, f->sel, f->nc, d_gv, f->radius,
                                     p->eval_prec, L, ws, (cudaStream_t)stream);
    if (s != RBF_OK)
        return s;
    return rbf_factor_solve(f, (const double *)(ws + L.gc), p->refine_steps, d_gc, h_max_resid,
                            stream);
}
