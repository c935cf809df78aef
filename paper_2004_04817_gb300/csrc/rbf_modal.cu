// rbf_modal.cu -- modal volume deformation on the 5th-generation tensor cores.
//
// Where k displacement fields (modes) share one support set, Eq. 6 for all
// of them is one product D = Phi_vc W with W of size N_c x n_out (n_out = 3 k
// columns).  Each CTA owns 128 volume points at a time (one M = 128 tile) and
// walks the centres in K-tiles of 64:
//   - sixteen warps evaluate phi (FP32): a thread takes two rows (points)
//     and one 8-centre chunk of the K-tile, and stores phi as BF16 in shared
//     memory in a K-major layout of 8 x 16-byte core matrices (no swizzle).
//     phi generation on the FP32 pipe is the bound of this kernel (about 20
//     instructions per pair against 192 MMA flops), so the CTA carries 16
//     warps, each thread with two independent chains, to hide the latency
//     of a pair's dependent chain;
//   - the matching K-tile of W (pre-packed in the same layout by an earlier
//     kernel) arrives by a bulk (TMA) copy completed on an mbarrier, started
//     one K-tile ahead; W buffers are touched only by the async proxy, so the
//     copies need no proxy fences;
//   - a seventeenth warp issues tcgen05.mma (kind::f16, BF16 x BF16 ->
//     FP32) with the accumulator in tensor memory.  The phi warps hand it
//     each finished A tile through an mbarrier (one arrival per warp), and it
//     commits each K-tile's MMAs to a second mbarrier that releases the
//     buffer; with two buffers, phi generation of tile t+1 overlaps the MMAs
//     of tile t and no block-wide barrier sits in the loop;
//   - four more warps (one per TMEM lane quarter) read the 128 x n_out FP32
//     accumulator with tcgen05.ld and store it; two accumulators in TMEM let
//     them drain tile t while the MMAs of tile t+1 run, so phi generation
//     never stops for the epilogue.
// Precision modes: BF16 (one product); BF16x3, where phi and W are split
// into three BF16 parts (x = x0 + x1 + x2, parts of order 1, 2^-9, 2^-18) and
// the six products down to order 2^-18 are accumulated (about FP32 accuracy);
// and FP16x2, where phi and the column-scaled W are split into two FP16
// parts (orders 1, 2^-11) and the three products x0 w0, x0 w1, x1 w0 are
// accumulated (FP16's 11-bit significand makes two parts as precise as three
// BF16 ones, at half the products).
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kMM = 128;          // points per tile (MMA M)
constexpr int kMK = 64;           // centres per K-tile
constexpr int kMProducers = 16;   // phi warps 0 .. 15
constexpr int kMEpilogue = 4;     // epilogue warps 17 .. 20 (TMEM lanes 32 (w mod 4) ..)
constexpr int kMThreads = 32 * (kMProducers + 1 + kMEpilogue);   // + warp 16: MMAs
constexpr int kModalMaxOut = 256; // MMA N limit
constexpr int kModalMaxCentres = 4096;

// byte offset of element (row, k) in a K-major no-swizzle tile of 8x8 core
// matrices (rows of 16 bytes), K extent kMK: core (row/8, k/8) at
// ((row/8) * (kMK/8) + k/8) * 128, then (row%8) * 16 + (k%8) * 2.  Used for
// W: descriptor LBO 128 (next core along K), SBO kMK/8 * 128 (next 8 rows).
__host__ __device__ __forceinline__ int kmajor_off(int row, int k)
{
    return ((row >> 3) * (kMK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// The A (phi) tile: the same core matrices with the 8-row groups adjacent,
// core (row/8, k/8) at (k/8) * kMM/8 * 128 + (row/8) * 128, i.e. each
// 8-centre chunk is a plane of kMM rows of 16 bytes.  Descriptor LBO
// kMM/8 * 128 = 2048 (next core along K), SBO 128 (next 8 rows).  A warp
// writing 32 consecutive rows of one chunk fills 512 contiguous bytes.
constexpr int kAPlane = kMM / 8 * 128;
__device__ __forceinline__ int a_off(int row, int k)
{
    return (k >> 3) * kAPlane + row * 16 + (k & 7) * 2;
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

// Instruction descriptor, kind::f16: D format F32 (bit 4), A and B of ONE
// type (bits 7-9 and 10-12: 1 = BF16, 0 = FP16, always set together), both
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ __forceinline__ uint32_t idesc_f16kind(int m, int n, bool fp16)
{
    const uint32_t fmt = fp16 ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
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

__device__ __forceinline__ unsigned bf2_bits(__nv_bfloat162 v)
{
    return *reinterpret_cast<unsigned *>(&v);
}

// Eight FP32 values to BF16 (round to nearest even), two per conversion.
__device__ __forceinline__ uint4 pack8_f(const float *x)
{
    uint4 r;
    r.x = bf2_bits(__floats2bfloat162_rn(x[0], x[1]));
    r.y = bf2_bits(__floats2bfloat162_rn(x[2], x[3]));
    r.z = bf2_bits(__floats2bfloat162_rn(x[4], x[5]));
    r.w = bf2_bits(__floats2bfloat162_rn(x[6], x[7]));
    return r;
}

// Three-way split of eight values, two per conversion: x = b0 + b1 + b2
// element by element, the same parts as split3.
__device__ __forceinline__ void split3_pack8(const float *x, uint4 &q0, uint4 &q1, uint4 &q2)
{
    unsigned o0[4], o1[4], o2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 b0 = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        const float2 f0 = __bfloat1622float2(b0);
        const float r0 = x[2 * i] - f0.x, r1 = x[2 * i + 1] - f0.y;
        const __nv_bfloat162 b1 = __floats2bfloat162_rn(r0, r1);
        const float2 f1 = __bfloat1622float2(b1);
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0 - f1.x, r1 - f1.y);
        o0[i] = bf2_bits(b0);
        o1[i] = bf2_bits(b1);
        o2[i] = bf2_bits(b2);
    }
    q0 = make_uint4(o0[0], o0[1], o0[2], o0[3]);
    q1 = make_uint4(o1[0], o1[1], o1[2], o1[3]);
    q2 = make_uint4(o2[0], o2[1], o2[2], o2[3]);
}

__device__ __forceinline__ unsigned h2_bits(__half2 v)
{
    return *reinterpret_cast<unsigned *>(&v);
}

// Two-way FP16 split of eight values in [0, 1], two per conversion:
// x = h0 + h1 element by element (h1 the nearest FP16 of x - h0).
__device__ __forceinline__ void split2_pack8_f16(const float *x, uint4 &q0, uint4 &q1)
{
    unsigned o0[4], o1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 h0 = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
        const float2 f0 = __half22float2(h0);
        const __half2 h1 = __floats2half2_rn(x[2 * i] - f0.x, x[2 * i + 1] - f0.y);
        o0[i] = h2_bits(h0);
        o1[i] = h2_bits(h1);
    }
    q0 = make_uint4(o0[0], o0[1], o0[2], o0[3]);
    q1 = make_uint4(o1[0], o1[1], o1[2], o1[3]);
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
    int tmem_cols;   // TMEM columns per accumulator (power of 2 >= its width)
    int pair;        // split modes with n_out <= 128: products x0 [w0|w1] (and, for
                     // BF16x3, x1 [w0|w1]) as N = 2 n_out MMAs into a 2 n_out
                     // accumulator whose halves the epilogue adds (BF16x3: 4
                     // MMAs per K step, not 6; FP16x2: 2, not 3)
    size_t a_bytes;  // one A tile (one split)
    size_t w_bytes;  // one W K-tile (one split)
    int nw;          // W K-tile buffers: 3 where shared memory allows, else 2
};

// bulk_g2s without the proxy fences, for a source written before the kernel
// started (the launch boundary orders it) into shared memory that only the
// async proxy touches (bulk copies write it, tcgen05.mma reads it).
__device__ __forceinline__ void bulk_g2s_static(void *dst, const void *src, unsigned bytes,
                                                unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase that also gives up once another thread
// of the CTA has raised the shared failure flag.
__device__ __forceinline__ bool mbar_wait_or_fail(unsigned long long *bar, unsigned parity,
                                                  uint64_t limit_ns, volatile int *fail)
{
    const unsigned a = smem_addr(bar);
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done)
            return true;
        if (*fail)
            return false;
        if (it == 0) {
            t0 = globaltimer_ns();
        } else if (globaltimer_ns() - t0 > limit_ns) {
            *fail = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Shared memory: [centres float4 x nc_pad][A buf0 x splits][A buf1 x splits]
//                [W buf0 .. buf nw-1, x splits each][11 mbarriers][tmem slot][fail flag]
// K-tiles are counted across the CTA's M tiles (g = 0, 1, ...); K-tile g uses
// A buffer g & 1 and W buffer g mod nw.  The CTA's i-th M tile accumulates in
// TMEM accumulator i & 1, which the epilogue warps drain while the MMAs of
// tile i + 1 fill the other.  Every mbarrier completes once per use of its
// buffer or accumulator, so use u waits for phase parity u & 1; no barrier
// can run two phases ahead of a waiter, because its next completion needs
// that waiter's own next step.
template <int SPLITS>
__global__ void __launch_bounds__(kMThreads, 1)
k_modal(const float4 *__restrict__ xq, int64_t nv, const float4 *__restrict__ centres,
        int nc_pad, const uint8_t *__restrict__ wpack, ModalShape sh, float *__restrict__ out,
        const float *__restrict__ wscale, int *status, uint64_t limit_ns)
{
    constexpr int kProd = SPLITS == 1 ? 1 : SPLITS == 2 ? 3 : 6;   // (phi part, W part) products
    constexpr bool kF16 = SPLITS == 2;   // FP16 parts (both operands), else BF16
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float4 *s_c = (float4 *)smem;
    uint8_t *s_a = smem + ((sizeof(float4) * (size_t)nc_pad + 1023) & ~(size_t)1023);
    uint8_t *s_w = s_a + 2 * sh.splits * sh.a_bytes;
    unsigned long long *bars = (unsigned long long *)(s_w + sh.nw * sh.splits * sh.w_bytes);
    // per W buffer: K-tile loaded; per A buffer: MMAs done, A tile written
    // (16 warps); per accumulator: tile's MMAs done, epilogue done (4 warps)
    unsigned long long *wfull = bars, *mdone = bars + 3, *afull = bars + 5;
    unsigned long long *accfull = bars + 7, *accfree = bars + 9;
    unsigned *s_tmem = (unsigned *)(bars + 11);
    volatile int *fail = (volatile int *)(s_tmem + 1);   // a wait gave up

    for (int j = tid; j < nc_pad; j += kMThreads)
        s_c[j] = centres[j];
    if (tid == 0) {
        *fail = 0;
        for (int i = 0; i < 3; ++i)
            mbar_init(&wfull[i], 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&mdone[i], 1);
            mbar_init(&afull[i], kMProducers);
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], kMEpilogue);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(s_tmem)),
                     "r"(2 * sh.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *s_tmem;
    const int64_t ntiles = (nv + kMM - 1) / kMM;

    if (warp == kMProducers) {
        // ---------------- MMA warp (lane 0) ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_f16kind(kMM, sh.n_out, kF16);
            const uint32_t idesc2 = idesc_f16kind(kMM, 2 * sh.n_out, kF16);   // pair mode
            const size_t wbytes = SPLITS * sh.w_bytes;
            // this CTA's K-tiles: its M tiles times nkt
            const long long gtot =
                (long long)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x) * sh.nkt;
            // descriptors of buffer pair 0; pair 1 and the parts of a split
            // are fixed address offsets (the start-address field holds
            // address / 16 and no sum leaves shared memory)
            const uint64_t ad0 = smem_desc(smem_addr(s_a), kAPlane, 128);
            const uint64_t wd0 = smem_desc(smem_addr(s_w), 128, (kMK / 8) * 128);
            const uint64_t a_buf = (uint64_t)(SPLITS * sh.a_bytes) >> 4;
            const uint64_t a_part = (uint64_t)sh.a_bytes >> 4;
            const uint64_t w_buf = (uint64_t)wbytes >> 4, w_part = (uint64_t)sh.w_bytes >> 4;
            long long g = 0;
            int i = 0;   // M tiles of this CTA
            int last_acc = -1;   // tile of the last accumulator commit
            bool ok = true;
            // W ring: K-tile j in buffer j mod nw.  Copies run ahead: with
            // three buffers W(g + 1) starts before K-tile g's MMAs (its
            // buffer was last read by the MMAs of g - 2); with two, after
            // them (its buffer was last read by those of g - 1).
            long long w_issued = 0;   // copies started: W(0) .. W(w_issued - 1)
            int wb = 0;               // buffer of K-tile g
            unsigned wpar = 0;        // bit b: parity of buffer b's next completion
            auto w_start = [&](long long j, int kt_j) {
                const int b = (int)(j % sh.nw);
                bulk_g2s_static(s_w + b * wbytes, wpack + (size_t)kt_j * wbytes, (unsigned)wbytes,
                                &wfull[b]);
                w_issued = j + 1;
            };
            if (gtot > 0)
                w_start(0, 0);
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
                const int ab = i & 1;
                // accumulator ab: free once tile i - 2's epilogue is done
                if (i >= 2 &&
                    !mbar_wait_or_fail(&accfree[ab], (unsigned)((i >> 1) - 1) & 1u, limit_ns,
                                       fail)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned dacc = tmem + (unsigned)(ab * sh.tmem_cols);
                for (int kt = 0; kt < sh.nkt; ++kt, ++g) {
                    const int buf = (int)(g & 1);
                    const unsigned par = (unsigned)(g >> 1) & 1u;
                    const int kt_next = kt + 1 == sh.nkt ? 0 : kt + 1;
                    if (sh.nw == 3 && g + 1 < gtot) {
                        if (g >= 2 && !mbar_wait_or_fail(&mdone[buf], par ^ 1u, limit_ns, fail)) {
                            ok = false;
                            break;
                        }
                        w_start(g + 1, kt_next);
                    }
                    if (!mbar_wait_or_fail(&wfull[wb], (wpar >> wb) & 1u, limit_ns, fail)) {
                        ok = false;
                        break;
                    }
                    wpar ^= 1u << wb;
                    if (!mbar_wait_or_fail(&afull[buf], par, limit_ns, fail)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ab_d = ad0 + (buf ? a_buf : 0), wb_d = wd0 + wb * w_buf;
                    if (SPLITS == 2 && sh.pair) {
                        // x0 [w0|w1] (N = 2 n_out) and x1 w0 (N = n_out)
#pragma unroll
                        for (int ks = 0; ks < kMK / 16; ++ks) {
                            const uint64_t ao = (uint64_t)(ks * 2 * kAPlane / 16);
                            const uint64_t wo = (uint64_t)(ks * 256 / 16);
                            mma_bf16(dacc, ab_d + ao, wb_d + wo, idesc2, (kt | ks) != 0);
                            mma_bf16(dacc, ab_d + a_part + ao, wb_d + wo, idesc, 1);
                        }
                    } else if (SPLITS == 3 && sh.pair) {
                        // x0 [w0|w1] and x1 [w0|w1] (N = 2 n_out; the W parts
                        // are adjacent along N), x0 w2 and x2 w0 (N = n_out)
#pragma unroll
                        for (int ks = 0; ks < kMK / 16; ++ks) {
                            const uint64_t ao = (uint64_t)(ks * 2 * kAPlane / 16);
                            const uint64_t wo = (uint64_t)(ks * 256 / 16);
                            mma_bf16(dacc, ab_d + ao, wb_d + wo, idesc2, (kt | ks) != 0);
                            mma_bf16(dacc, ab_d + a_part + ao, wb_d + wo, idesc2, 1);
                            mma_bf16(dacc, ab_d + ao, wb_d + 2 * w_part + wo, idesc, 1);
                            mma_bf16(dacc + (unsigned)sh.n_out, ab_d + 2 * a_part + ao, wb_d + wo,
                                     idesc, 1);
                        }
                    } else {
#pragma unroll
                        for (int pr = 0; pr < kProd; ++pr) {
                            // products x0 w0, x0 w1, x1 w0, x0 w2, x1 w1, x2 w0
                            // (FP16x2: the first three)
                            const int ia =
                                SPLITS == 1 ? 0 : (pr == 2 || pr == 4) ? 1 : pr == 5 ? 2 : 0;
                            const int iw = SPLITS == 1 ? 0 : pr == 1 || pr == 4 ? 1 : pr == 3 ? 2 : 0;
#pragma unroll
                            for (int ks = 0; ks < kMK / 16; ++ks) {
                                // K step of 16 = two core matrices along K: A at
                                // 2 x kAPlane bytes, W at 256 bytes
                                const uint64_t ad =
                                    ab_d + ia * a_part + (uint64_t)(ks * 2 * kAPlane / 16);
                                const uint64_t bd = wb_d + iw * w_part + (uint64_t)(ks * 256 / 16);
                                mma_bf16(dacc, ad, bd, idesc, (kt | pr | ks) != 0);
                            }
                        }
                    }
                    mma_commit(&mdone[buf]);
                    if (sh.nw == 2 && g + 1 < gtot) {
                        if (g >= 1 && !mbar_wait_or_fail(&mdone[buf ^ 1],
                                                         (unsigned)((g - 1) >> 1) & 1u, limit_ns,
                                                         fail)) {
                            ok = false;
                            break;
                        }
                        w_start(g + 1, kt_next);
                    }
                    wb = wb + 1 == sh.nw ? 0 : wb + 1;
                }
                if (ok) {
                    mma_commit(&accfull[ab]);
                    last_acc = i;
                }
            }
            // nothing of this thread in flight at exit: the W copies started
            // but not waited for (W(g) .. W(w_issued - 1); K-tile g's own wait
            // may have given up), and the arrivals of the last commits
            for (long long j = g; j < w_issued; ++j)
                mbar_wait(&wfull[j % sh.nw], (unsigned)(j / sh.nw) & 1u, limit_ns);
            if (g >= 1)
                mbar_wait(&mdone[(g - 1) & 1], (unsigned)((g - 1) >> 1) & 1u, limit_ns);
            if (last_acc >= 0)
                mbar_wait(&accfull[last_acc & 1], (unsigned)(last_acc >> 1) & 1u, limit_ns);
        }
    } else if (warp < kMProducers) {
        // ---------------- phi warps ----------------
        // rows 64 (warp mod 2) + lane and + 32 + lane of the tile, 8-centre
        // chunk warp / 2 of each K-tile: every lane of a warp reads the same
        // centre (a broadcast) for two independent phi chains, and a warp's
        // stores fill 512 contiguous bytes per row set
        const int row0 = (warp & 1) * 64 + lane, row1 = row0 + 32;
        const int chunk = warp >> 1;
        long long g = 0;
        bool ok = true;
        auto point = [&](int64_t t, int row) {
            int64_t v = t * kMM + row;
            v = v < nv ? v : nv - 1;
            return xq[v];
        };
        float4 q0n = point(blockIdx.x, row0), q1n = point(blockIdx.x, row1);
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const float4 q0 = q0n, q1 = q1n;
            const f2 qx2 = f2_pack(q0.x, q1.x), qy2 = f2_pack(q0.y, q1.y),
                     qz2 = f2_pack(q0.z, q1.z);
            if (tile + gridDim.x < ntiles) {   // in flight during this tile
                q0n = point(tile + gridDim.x, row0);
                q1n = point(tile + gridDim.x, row1);
            }
            for (int kt = 0; kt < sh.nkt; ++kt, ++g) {
                const int buf = (int)(g & 1);
                const unsigned par = (unsigned)(g >> 1) & 1u;
                // the A buffer: free once the MMAs of use g - 2 are done
                if (g >= 2 && !mbar_wait_or_fail(&mdone[buf], par ^ 1u, limit_ns, fail)) {
                    ok = false;
                    break;
                }
                uint8_t *a0 = s_a + buf * SPLITS * sh.a_bytes;
                const int k8 = 8 * chunk;
                // both rows at once on the paired FP32 pipe (same operations
                // and rounding as the scalar path, one instruction for two)
                float ph0[8], ph1[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const float4 c = s_c[kt * kMK + k8 + kk];
                    const f2 dx = f2_sub(qx2, f2_bcast(c.x)), dy = f2_sub(qy2, f2_bcast(c.y)),
                             dz = f2_sub(qz2, f2_bcast(c.z));
                    const f2 ph = phi_f32x2_s(f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx))));
                    f2_unpack(ph, ph0[kk], ph1[kk]);
                }
                const int off0 = a_off(row0, k8), off1 = a_off(row1, k8);
                if (SPLITS == 1) {
                    *(uint4 *)(a0 + off0) = pack8_f(ph0);
                    *(uint4 *)(a0 + off1) = pack8_f(ph1);
                } else if (SPLITS == 2) {
                    uint4 u0, u1;
                    split2_pack8_f16(ph0, u0, u1);
                    *(uint4 *)(a0 + off0) = u0;
                    *(uint4 *)(a0 + sh.a_bytes + off0) = u1;
                    split2_pack8_f16(ph1, u0, u1);
                    *(uint4 *)(a0 + off1) = u0;
                    *(uint4 *)(a0 + sh.a_bytes + off1) = u1;
                } else {
                    uint4 u0, u1, u2;
                    split3_pack8(ph0, u0, u1, u2);
                    *(uint4 *)(a0 + off0) = u0;
                    *(uint4 *)(a0 + sh.a_bytes + off0) = u1;
                    *(uint4 *)(a0 + 2 * sh.a_bytes + off0) = u2;
                    split3_pack8(ph1, u0, u1, u2);
                    *(uint4 *)(a0 + off1) = u0;
                    *(uint4 *)(a0 + sh.a_bytes + off1) = u1;
                    *(uint4 *)(a0 + 2 * sh.a_bytes + off1) = u2;
                }
                // generic-proxy stores -> visible to the tensor core (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&afull[buf]);
            }
        }
    } else {
        // ---------------- epilogue warps ----------------
        // the CTA's tile i: accumulator i & 1, TMEM lanes 32 (warp mod 4) ..
        // +31 (rows of the tile), every 32-column group
        const int quarter = warp & 3;
        int i = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            if (!mbar_wait_or_fail(&accfull[i & 1], (unsigned)(i >> 1) & 1u, limit_ns, fail))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t ev = tile * kMM + quarter * 32 + lane;
            float *orow = out + (size_t)(ev < nv ? ev : 0) * sh.n_out;
            const unsigned lane_base =
                tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)((i & 1) * sh.tmem_cols);
            // FP16x2: each column's power-of-two scale of W, undone here
            auto scl = [&](int col) { return SPLITS == 2 ? __ldg(wscale + col) : 1.0f; };
            if (sh.pair) {
                // the two halves of the accumulator, 16 columns at a time
                for (int c0 = 0; c0 < sh.n_out; c0 += 16) {
                    float lo[16], hi[16];
                    tmem_ld16(lane_base + (unsigned)c0, lo);
                    tmem_ld16(lane_base + (unsigned)(c0 + sh.n_out), hi);
                    if (ev < nv) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            *(float4 *)(orow + c0 + e) =
                                make_float4((lo[e] + hi[e]) * scl(c0 + e),
                                            (lo[e + 1] + hi[e + 1]) * scl(c0 + e + 1),
                                            (lo[e + 2] + hi[e + 2]) * scl(c0 + e + 2),
                                            (lo[e + 3] + hi[e + 3]) * scl(c0 + e + 3));
                    }
                }
            } else {
                for (int c0 = 0; c0 < sh.n_out; c0 += 32) {
                    if (c0 + 32 <= sh.n_out) {
                        float vals[32];
                        tmem_ld32(lane_base + (unsigned)c0, vals);
                        if (ev < nv) {
#pragma unroll
                            for (int e = 0; e < 32; e += 4)
                                *(float4 *)(orow + c0 + e) = make_float4(
                                    vals[e] * scl(c0 + e), vals[e + 1] * scl(c0 + e + 1),
                                    vals[e + 2] * scl(c0 + e + 2), vals[e + 3] * scl(c0 + e + 3));
                        }
                    } else {   // n_out % 32 == 16: one 16-column tail
                        float vals[16];
                        tmem_ld16(lane_base + (unsigned)c0, vals);
                        if (ev < nv) {
#pragma unroll
                            for (int e = 0; e < 16; e += 4)
                                *(float4 *)(orow + c0 + e) = make_float4(
                                    vals[e] * scl(c0 + e), vals[e + 1] * scl(c0 + e + 1),
                                    vals[e + 2] * scl(c0 + e + 2), vals[e + 3] * scl(c0 + e + 3));
                        }
                    }
                }
            }
            // the TMEM reads are done before the accumulator is handed back
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&accfree[i & 1]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*fail && tid == 0)
        atomicExch(status, (int)RBF_E_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * sh.tmem_cols)
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

// FP16x2: per column c of W, the power of two 2^(e+1) with max_j |W_jc| <
// 2^(e+1), so that W / scale lies in (-1, 1) (1 for an all-zero column).
// One thread per column (n_out <= 256).
__global__ void k_modal_col_scale(const double *__restrict__ W, int nc, int n_out,
                                  float *__restrict__ scale)
{
    const int c = threadIdx.x;
    if (c >= n_out)
        return;
    double m = 0.0;
    for (int j = 0; j < nc; ++j)
        m = fmax(m, fabs(W[(size_t)j * n_out + c]));
    scale[c] = m > 0.0 ? (float)ldexp(1.0, ilogb(m) + 1) : 1.0f;
}

__global__ void k_modal_pack_w(const double *__restrict__ W, int nc, int n_out, int nkt,
                               int splits, size_t w_bytes, const float *__restrict__ scale,
                               uint8_t *__restrict__ wpack)
{
    const int64_t total = (int64_t)nkt * kMK * n_out;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(t % n_out);
        const int64_t kg = t / n_out;          // global centre index
        const int kt = (int)(kg / kMK), k = (int)(kg % kMK);
        uint8_t *base = wpack + (size_t)kt * splits * w_bytes;
        const int off = kmajor_off(n, k);
        if (splits == 2) {   // FP16 parts of W / scale (power of two: exact)
            const float x = kg < nc ? (float)(W[kg * n_out + n] / (double)scale[n]) : 0.0f;
            const __half h0 = __float2half_rn(x);
            const __half h1 = __float2half_rn(x - __half2float(h0));
            *(__half *)(base + off) = h0;
            *(__half *)(base + w_bytes + off) = h1;
            continue;
        }
        const float x = kg < nc ? (float)W[kg * n_out + n] : 0.0f;
        __nv_bfloat16 b0, b1, b2;
        if (splits == 1) {
            b0 = __float2bfloat16_rn(x);
            b1 = b2 = b0;
        } else {
            split3(x, b0, b1, b2);
        }
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
    s.pair = splits > 1 && n_out <= 128;
    s.tmem_cols = 32;
    while (s.tmem_cols < (s.pair ? 2 : 1) * n_out)
        s.tmem_cols *= 2;
    s.a_bytes = (size_t)kMM * kMK * 2;
    s.w_bytes = (size_t)n_out * kMK * 2;
    s.nw = 2;
    return s;
}

static size_t modal_smem(const ModalShape &s)
{
    const size_t nc_pad = (size_t)s.nkt * kMK;
    return align_up(sizeof(float4) * nc_pad, 1024) + 2 * s.splits * s.a_bytes +
           (size_t)s.nw * s.splits * s.w_bytes + 11 * 8 + 16;
}

struct ModalWs {
    size_t status, xq, c, w, scale, total;
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
    L.scale = take(sizeof(float) * kModalMaxOut);
    L.total = o;
    return L;
}

}  // namespace rbf

using namespace rbf;

extern "C" size_t rbf_modal_workspace_bytes(int64_t nv, int64_t nc, int n_out, int mode)
{
    if (nv < 0 || nc < 1 || nc > kModalMaxCentres || n_out < 16 || n_out > kModalMaxOut ||
        n_out % 16 != 0 ||
        (mode != RBF_MODAL_BF16 && mode != RBF_MODAL_F16X2 && mode != RBF_MODAL_BF16X3))
        return 0;
    return modal_ws(nv, modal_shape(nc, n_out, mode)).total;
}

extern "C" rbf_status rbf_deform_modal(const double *d_xv, int64_t nv, const double *d_xb,
                                       const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                                       int n_out, const rbf_params *p, int mode, float *d_out,
                                       void *d_ws, size_t ws_bytes, void *stream)
{
    if (!p || !(p->radius > 0.0) || nv < 0 || nc < 1 || nc > kModalMaxCentres || n_out < 16 ||
        n_out > kModalMaxOut || n_out % 16 != 0 ||
        (mode != RBF_MODAL_BF16 && mode != RBF_MODAL_F16X2 && mode != RBF_MODAL_BF16X3))
        return RBF_E_ARG;
    if (nv == 0)
        return RBF_OK;
    if (!d_xv || !d_xb || !d_sel_idx || !d_w || !d_out || ((uintptr_t)d_out & 15) != 0)
        return RBF_E_ARG;
    ModalShape sh = modal_shape(nc, n_out, mode);   // mode = number of parts
    const ModalWs L = modal_ws(nv, sh);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    cudaFuncAttributes fattr{};
    const void *kfn = sh.splits == 1   ? (const void *)k_modal<1>
                      : sh.splits == 2 ? (const void *)k_modal<2>
                                       : (const void *)k_modal<3>;
    if (cudaFuncGetAttributes(&fattr, kfn) != cudaSuccess)
        return RBF_E_CUDA;
    ModalShape sh3 = sh;
    sh3.nw = 3;
    if (modal_smem(sh3) + fattr.sharedSizeBytes <= dev.smem_optin)
        sh = sh3;   // a third W buffer lets each copy start one K-tile earlier
    const size_t smem = modal_smem(sh);
    if (smem + fattr.sharedSizeBytes > dev.smem_optin)
        return RBF_E_ARG;   // too many centres or columns for the shared buffers
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    float4 *xq = (float4 *)(ws + L.xq);
    float4 *c = (float4 *)(ws + L.c);
    uint8_t *wp = (uint8_t *)(ws + L.w);
    float *wscale = (float *)(ws + L.scale);
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
    if (sh.splits == 2)
        k_modal_col_scale<<<1, kModalMaxOut, 0, st>>>(d_w, (int)nc, n_out, wscale);
    k_modal_pack_w<<<(int)std::min<int64_t>((wtot + 255) / 256, dev.sms * 8), 256, 0, st>>>(
        d_w, (int)nc, n_out, sh.nkt, sh.splits, sh.w_bytes, wscale, wp);
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RBF_E_CUDA;
    const int64_t ntiles = (nv + kMM - 1) / kMM;
    const int grid = (int)std::min<int64_t>(ntiles, dev.sms);
    if (sh.splits == 1)
        k_modal<1><<<grid, kMThreads, smem, st>>>(xq, nv, c, nc_pad, wp, sh, d_out, wscale,
                                                  status, kBarrierLimitNs);
    else if (sh.splits == 2)
        k_modal<2><<<grid, kMThreads, smem, st>>>(xq, nv, c, nc_pad, wp, sh, d_out, wscale,
                                                  status, kBarrierLimitNs);
    else
        k_modal<3><<<grid, kMThreads, smem, st>>>(xq, nv, c, nc_pad, wp, sh, d_out, wscale,
                                                  status, kBarrierLimitNs);
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
