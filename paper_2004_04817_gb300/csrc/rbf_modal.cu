// rbf_modal.cu -- modal volume deformation on the 5th-generation tensor cores.
//
// Where k displacement fields (modes) share one support set, Eq. 6 for all
// of them is one product D = Phi_vc W with W of size N_c x n_out (n_out = 3 k
// columns).  Each CTA owns 128 volume points at a time (one M = 128 tile) and
// walks the centres in K-tiles of 64:
//   - sixteen warps evaluate phi (FP32): thread t takes row t % 128 and 16
//     of the K-tile's 64 centres, and stores phi as BF16 in shared memory in
//     the canonical K-major layout (8 x 16-byte core matrices, no swizzle).
//     phi generation on the FP32 pipe is the bound of this kernel (about 20
//     instructions per pair against 192 MMA flops), so the CTA carries 16
//     warps to hide the latency of each pair's dependent chain;
//   - the matching K-tile of W (pre-packed in the same layout) arrives by a
//     bulk (TMA) copy completed on an mbarrier;
//   - one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) with
//     the accumulator in tensor memory and commits to an mbarrier; two
//     buffers let phi generation of tile t+1 overlap the MMAs of tile t, and
//     one block barrier per K-tile hands the finished A tile to the MMA
//     thread;
//   - the epilogue reads the 128 x n_out FP32 accumulator with tcgen05.ld
//     (warp w: TMEM lanes 32 (w mod 4) .. +31, column groups w / 4, w / 4 + 4,
//     ...) and stores it.
// Precision modes: BF16 (one product) and BF16x3, where phi and W are split
// into three BF16 parts (x = x0 + x1 + x2, parts of order 1, 2^-9, 2^-18) and
// the six products down to order 2^-18 are accumulated (about FP32 accuracy).
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kMM = 128;          // points per tile (MMA M)
constexpr int kMK = 64;           // centres per K-tile
constexpr int kMThreads = 512;    // sixteen warps; warp w reads TMEM lanes 32 (w mod 4) ..
constexpr int kModalMaxOut = 256; // MMA N limit
constexpr int kModalMaxCentres = 4096;

// byte offset of element (row, k) in a K-major no-swizzle tile of 8x8 core
// matrices (rows of 16 bytes), K extent kMK: core (row/8, k/8) at
// ((row/8) * (kMK/8) + k/8) * 128, then (row%8) * 16 + (k%8) * 2
__host__ __device__ __forceinline__ int kmajor_off(int row, int k)
{
    return ((row >> 3) * (kMK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor (tcgen05): start address >> 4 in bits 0-13,
// leading-dimension byte offset >> 4 in 16-29 (K direction: next core matrix
// along K), stride byte offset >> 4 in 32-45 (next 8-row group), descriptor
// version 1 in bits 46-47, no swizzle (layout 0 in bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D format F32 (bit 4), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float *v)
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 *b)
{
    uint4 r;
    r.x = (uint32_t)__bfloat16_as_ushort(b[0]) | ((uint32_t)__bfloat16_as_ushort(b[1]) << 16);
    r.y = (uint32_t)__bfloat16_as_ushort(b[2]) | ((uint32_t)__bfloat16_as_ushort(b[3]) << 16);
    r.z = (uint32_t)__bfloat16_as_ushort(b[4]) | ((uint32_t)__bfloat16_as_ushort(b[5]) << 16);
    r.w = (uint32_t)__bfloat16_as_ushort(b[6]) | ((uint32_t)__bfloat16_as_ushort(b[7]) << 16);
    return r;
}

// Three-way BF16 split: x = b0 + b1 + b2 (each the nearest BF16 of what is
// left), about 24 significant bits in all.
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &b0, __nv_bfloat16 &b1,
                                       __nv_bfloat16 &b2)
{
    b0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(b0);
    b1 = __float2bfloat16_rn(r1);
    b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
}

struct ModalShape {
    int n_out;       // columns (multiple of 16, <= 256)
    int nkt;         // K-tiles
    int splits;      // 1 (BF16) or 3 (BF16x3)
    int tmem_cols;   // allocated TMEM columns (power of 2 >= n_out)
    size_t a_bytes;  // one A tile (one split)
    size_t w_bytes;  // one W K-tile (one split)
};

// A product list for the split mode: (phi part, W part) pairs.
__constant__ int c_prod_a[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_prod_w[6] = {0, 1, 0, 2, 1, 0};

// Shared memory: [centres float4 x nc_pad][A buf0 x splits][A buf1 x splits]
//                [W buf0 x splits][W buf1 x splits][mbarriers][tmem slot]
__global__ void __launch_bounds__(kMThreads, 1)
k_modal(const float4 *__restrict__ xq, int64_t nv, const float4 *__restrict__ centres,
        int nc_pad, const uint8_t *__restrict__ wpack, ModalShape sh, float *__restrict__ out,
        int *status, uint64_t limit_ns)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    float4 *s_c = (float4 *)smem;
    uint8_t *s_a = smem + ((sizeof(float4) * (size_t)nc_pad + 1023) & ~(size_t)1023);
    uint8_t *s_w = s_a + 2 * sh.splits * sh.a_bytes;
    unsigned long long *bars = (unsigned long long *)(s_w + 2 * sh.splits * sh.w_bytes);
    // bars[0..1]: W tile loaded (per buffer); bars[2..3]: MMAs of buffer done
    unsigned *s_tmem = (unsigned *)(bars + 4);

    for (int j = tid; j < nc_pad; j += kMThreads)
        s_c[j] = centres[j];
    if (tid == 0) {
        for (int i = 0; i < 4; ++i)
            mbar_init(&bars[i], 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(s_tmem)),
                     "r"(sh.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *s_tmem;
    const uint32_t idesc = idesc_bf16(kMM, sh.n_out);
    unsigned wphase[2] = {0, 0}, mphase[2] = {0, 0};
    bool pending[2] = {false, false};
    bool ok = true;

    const int64_t ntiles = (nv + kMM - 1) / kMM;
    const int row = tid & (kMM - 1), kgrp = tid >> 7;   // kgrp: centres 16 kgrp .. +15
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int64_t v = tile * kMM + row;
        const bool live = v < nv;
        v = live ? v : nv - 1;
        const float4 q = xq[v];
        for (int kt = 0; kt < sh.nkt; ++kt) {
            const int buf = kt & 1;
            bool mine = true;
            // the MMAs that last read this buffer pair must be done
            if (pending[buf]) {
                mine = mbar_wait(&bars[2 + buf], mphase[buf], limit_ns);
                if (mine) {   // else the exit path waits again for the MMAs in flight
                    mphase[buf] ^= 1u;
                    pending[buf] = false;
                }
            }
            // W K-tile (all splits) by one bulk copy
            if (tid == 0 && mine) {
                const size_t bytes = sh.splits * sh.w_bytes;
                bulk_g2s(s_w + buf * sh.splits * sh.w_bytes, wpack + (size_t)kt * bytes,
                         (unsigned)bytes, &bars[buf]);
            }
            // phi for this thread's row and its 16 centres of the K-tile
            uint8_t *a0 = s_a + buf * sh.splits * sh.a_bytes;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k8 = kgrp * 16 + h * 8;
                __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const float4 c = s_c[kt * kMK + k8 + kk];
                    const float dx = q.x - c.x, dy = q.y - c.y, dz = q.z - c.z;
                    const float ph = phi_f32_s(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                    if (sh.splits == 1) {
                        p0[kk] = __float2bfloat16_rn(ph);
                    } else {
                        split3(ph, p0[kk], p1[kk], p2[kk]);
                    }
                }
                const int off = kmajor_off(row, k8);
                *(uint4 *)(a0 + off) = pack8(p0);
                if (sh.splits == 3) {
                    *(uint4 *)(a0 + sh.a_bytes + off) = pack8(p1);
                    *(uint4 *)(a0 + 2 * sh.a_bytes + off) = pack8(p2);
                }
            }
            // generic-proxy stores -> visible to the tensor core (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            // one barrier: the A tile is complete, and every thread learns
            // whether a wait anywhere in the CTA gave up
            if (__syncthreads_or(!mine || *(volatile int *)status == (int)RBF_E_TIMEOUT)) {
                ok = false;
                break;
            }
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool got = mbar_wait(&bars[buf], wphase[buf], limit_ns);
                wphase[buf] ^= 1u;
                if (!got) {
                    atomicExch(status, (int)RBF_E_TIMEOUT);
                } else {
                    const uint8_t *w0 = s_w + buf * sh.splits * sh.w_bytes;
                    const int nprod = sh.splits == 1 ? 1 : 6;
                    for (int pr = 0; pr < nprod; ++pr) {
                        const int ia = sh.splits == 1 ? 0 : c_prod_a[pr];
                        const int iw = sh.splits == 1 ? 0 : c_prod_w[pr];
                        const unsigned abase = smem_addr(a0 + ia * sh.a_bytes);
                        const unsigned wbase = smem_addr(w0 + iw * sh.w_bytes);
#pragma unroll
                        for (int ks = 0; ks < kMK / 16; ++ks) {
                            // K step of 16 = two core matrices along K (256 bytes)
                            const uint64_t ad = smem_desc(abase + ks * 256, 128, (kMK / 8) * 128);
                            const uint64_t bd = smem_desc(wbase + ks * 256, 128, (kMK / 8) * 128);
                            mma_bf16(tmem, ad, bd, idesc, (kt | pr | ks) != 0);
                        }
                    }
                    mma_commit(&bars[2 + buf]);
                }
            }
            pending[buf] = true;
        }
        // accumulator complete once the last commit has landed
        bool mine = ok;
        for (int b = 0; b < 2 && mine; ++b) {
            if (pending[b]) {
                mine = mbar_wait(&bars[2 + b], mphase[b], limit_ns);
                if (mine) {
                    mphase[b] ^= 1u;
                    pending[b] = false;
                }
            }
        }
        if (__syncthreads_or(!mine || !ok || *(volatile int *)status == (int)RBF_E_TIMEOUT)) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +31 (rows of the
        // tile) and the 32-column groups w / 4, w / 4 + 4, ...
        const int quarter = warp & 3;
        const int erow = quarter * 32 + (tid & 31);
        const int64_t ev = tile * kMM + erow;
        float *orow = out + (size_t)(ev < nv ? ev : 0) * sh.n_out;
        const unsigned lane_base = tmem + ((unsigned)(quarter * 32) << 16);
        for (int c0 = (warp >> 2) * 32; c0 < sh.n_out; c0 += 128) {
            if (c0 + 32 <= sh.n_out) {
                float vals[32];
                tmem_ld32(lane_base + (unsigned)c0, vals);
                if (ev < nv) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        *(float4 *)(orow + c0 + i) =
                            make_float4(vals[i], vals[i + 1], vals[i + 2], vals[i + 3]);
                }
            } else {   // n_out % 32 == 16: one 16-column tail
                float vals[16];
                tmem_ld16(lane_base + (unsigned)c0, vals);
                if (ev < nv) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *(float4 *)(orow + c0 + i) =
                            make_float4(vals[i], vals[i + 1], vals[i + 2], vals[i + 3]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok) {
        // leave nothing in flight: bounded waits for outstanding work
        for (int b = 0; b < 2; ++b) {
            if (pending[b])
                mbar_wait(&bars[2 + b], mphase[b], limit_ns);
        }
        if (tid == 0)
            atomicExch(status, (int)RBF_E_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(sh.tmem_cols)
                     : "memory");
}

// Packing: points scaled to float4; centres scaled (padding far away, phi 0);
// W split into BF16 parts in the K-major core-matrix layout, one K-tile
// (all splits) contiguous: [kt][split][n_out x kMK].
__global__ void k_modal_pack_centres(const double *__restrict__ xb,
                                     const int32_t *__restrict__ sel, int nc, int nc_pad,
                                     double inv_r, float4 *__restrict__ c)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc_pad; j += gridDim.x * blockDim.x) {
        if (j < nc) {
            const int64_t n = sel[j];
            c[j] = make_float4((float)(xb[3 * n] * inv_r), (float)(xb[3 * n + 1] * inv_r),
                               (float)(xb[3 * n + 2] * inv_r), 0.0f);
        } else {
            c[j] = make_float4(1e6f, 1e6f, 1e6f, 0.0f);   // beyond every support radius
        }
    }
}

__global__ void k_modal_pack_w(const double *__restrict__ W, int nc, int n_out, int nkt,
                               int splits, size_t w_bytes, uint8_t *__restrict__ wpack)
{
    const int64_t total = (int64_t)nkt * kMK * n_out;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(t % n_out);
        const int64_t kg = t / n_out;          // global centre index
        const int kt = (int)(kg / kMK), k = (int)(kg % kMK);
        const float x = kg < nc ? (float)W[kg * n_out + n] : 0.0f;
        __nv_bfloat16 b0, b1, b2;
        if (splits == 1) {
            b0 = __float2bfloat16_rn(x);
            b1 = b2 = b0;
        } else {
            split3(x, b0, b1, b2);
        }
        uint8_t *base = wpack + (size_t)kt * splits * w_bytes;
        const int off = kmajor_off(n, k);
        *(__nv_bfloat16 *)(base + off) = b0;
        if (splits == 3) {
            *(__nv_bfloat16 *)(base + w_bytes + off) = b1;
            *(__nv_bfloat16 *)(base + 2 * w_bytes + off) = b2;
        }
    }
}

__global__ void k_modal_pack_points(const double *__restrict__ x, int64_t n, double inv_r,
                                    float4 *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float4((float)(x[3 * i] * inv_r), (float)(x[3 * i + 1] * inv_r),
                             (float)(x[3 * i + 2] * inv_r), 0.0f);
}

static ModalShape modal_shape(int64_t nc, int n_out, int splits)
{
    ModalShape s{};
    s.n_out = n_out;
    s.nkt = (int)((nc + kMK - 1) / kMK);
    s.splits = splits;
    s.tmem_cols = 32;
    while (s.tmem_cols < n_out)
        s.tmem_cols *= 2;
    s.a_bytes = (size_t)kMM * kMK * 2;
    s.w_bytes = (size_t)n_out * kMK * 2;
    return s;
}

static size_t modal_smem(const ModalShape &s)
{
    const size_t nc_pad = (size_t)s.nkt * kMK;
    return align_up(sizeof(float4) * nc_pad, 1024) + 2 * s.splits * s.a_bytes +
           2 * s.splits * s.w_bytes + 4 * 8 + 16;
}

struct ModalWs {
    size_t status, xq, c, w, total;
};

static ModalWs modal_ws(int64_t nv, const ModalShape &s)
{
    ModalWs L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.status = take(sizeof(int));
    L.xq = take(sizeof(float4) * (size_t)nv);
    L.c = take(sizeof(float4) * (size_t)s.nkt * kMK);
    L.w = take((size_t)s.nkt * s.splits * s.w_bytes);
    L.total = o;
    return L;
}

}  // namespace rbf

using namespace rbf;

extern "C" size_t rbf_modal_workspace_bytes(int64_t nv, int64_t nc, int n_out, int mode)
{
    if (nv < 0 || nc < 1 || nc > kModalMaxCentres || n_out < 16 || n_out > kModalMaxOut ||
        n_out % 16 != 0 || (mode != RBF_MODAL_BF16 && mode != RBF_MODAL_BF16X3))
        return 0;
    return modal_ws(nv, modal_shape(nc, n_out, mode == RBF_MODAL_BF16 ? 1 : 3)).total;
}

extern "C" rbf_status rbf_deform_modal(const double *d_xv, int64_t nv, const double *d_xb,
                                       const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                                       int n_out, const rbf_params *p, int mode, float *d_out,
                                       void *d_ws, size_t ws_bytes, void *stream)
{
    if (!p || !(p->radius > 0.0) || nv < 0 || nc < 1 || nc > kModalMaxCentres || n_out < 16 ||
        n_out > kModalMaxOut || n_out % 16 != 0 ||
        (mode != RBF_MODAL_BF16 && mode != RBF_MODAL_BF16X3))
        return RBF_E_ARG;
    if (nv == 0)
        return RBF_OK;
    if (!d_xv || !d_xb || !d_sel_idx || !d_w || !d_out || ((uintptr_t)d_out & 15) != 0)
        return RBF_E_ARG;
    const ModalShape sh = modal_shape(nc, n_out, mode == RBF_MODAL_BF16 ? 1 : 3);
    const ModalWs L = modal_ws(nv, sh);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    const size_t smem = modal_smem(sh);
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    if (smem > dev.smem_optin)
        return RBF_E_ARG;   // too many centres for the resident centre table
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    float4 *xq = (float4 *)(ws + L.xq);
    float4 *c = (float4 *)(ws + L.c);
    uint8_t *wp = (uint8_t *)(ws + L.w);
    int *status = (int *)(ws + L.status);
    const double inv_r = 1.0 / p->radius;
    const int nc_pad = sh.nkt * kMK;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        return RBF_E_CUDA;
    k_modal_pack_points<<<(int)std::min<int64_t>((nv + 255) / 256, dev.sms * 8), 256, 0, st>>>(
        d_xv, nv, inv_r, xq);
    k_modal_pack_centres<<<(nc_pad + 127) / 128, 128, 0, st>>>(d_xb, d_sel_idx, (int)nc, nc_pad,
                                                              inv_r, c);
    const int64_t wtot = (int64_t)nc_pad * n_out;
    k_modal_pack_w<<<(int)std::min<int64_t>((wtot + 255) / 256, dev.sms * 8), 256, 0, st>>>(
        d_w, (int)nc, n_out, sh.nkt, sh.splits, sh.w_bytes, wp);
    if (cudaFuncSetAttribute(k_modal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RBF_E_CUDA;
    const int64_t ntiles = (nv + kMM - 1) / kMM;
    const int grid = (int)std::min<int64_t>(ntiles, dev.sms);
    k_modal<<<grid, kMThreads, smem, st>>>(xq, nv, c, nc_pad, wp, sh, d_out, status,
                                           kBarrierLimitNs);
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    return RBF_OK;
}

extern "C" rbf_status rbf_modal_check(const void *d_ws, void *stream)
{
    if (!d_ws)
        return RBF_E_ARG;
    int st = 0;
    if (cudaMemcpyAsync(&st, d_ws, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    return (rbf_status)st;
}
