// rbf_device.cuh -- device helpers shared by the librbfgcb kernels.
//
// Wendland C2 basis (Eq. 2 of arXiv:2004.04817) in FP32 and FP64, argmax key
// packing, and the bounded grid barrier used by the persistent kernels.
#pragma once

#include <cstdint>
#include <cstring>
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
// Paired FP32: two independent FP32 values in one 64-bit register, operated on
// by the f32x2 instructions of sm_100-class GPUs (one instruction, two
// results, each rounded to nearest like its scalar counterpart).
// ----------------------------------------------------------------------------
struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// Eq. 2 for two pairs at once, from their squared scaled distances s:
// s is clamped to 1 (so eta <= 1 and phi = 0 beyond the support radius), then
// t = 1 - eta, phi = t^4 (4 eta + 1) -- the factored form, whose rounding
// error stays proportional to |phi'| |d eta|.
__device__ __forceinline__ f2 phi_f32x2_s(f2 s)
{
    float s0, s1;
    f2_unpack(s, s0, s1);
    const f2 eta = f2_pack(sqrt_approx(fminf(s0, 1.0f)), sqrt_approx(fminf(s1, 1.0f)));
    const f2 one = f2_pack(1.0f, 1.0f), four = f2_pack(4.0f, 4.0f);
    const f2 t = f2_sub(one, eta);
    const f2 t2 = f2_mul(t, t);
    return f2_mul(f2_mul(t2, t2), f2_fma(four, eta, one));
}

// ----------------------------------------------------------------------------
// Double-float ("ff") arithmetic on the FP32 pipe: a value is the unevaluated
// sum h + l of two floats (about 48 significant bits).  Built from the
// error-free transformations of Knuth (TwoSum: the exact rounding error of a
// sum) and Dekker (FastTwoSum for |a| >= |b|; the exact error of a product
// through one fused multiply-add).  The __f*_rn intrinsics keep the compiler
// from contracting or reordering the steps whose rounding the method needs.
// On GB300 an ff pair costs ~110 FP32 instructions (paired), 20x less time than the
// same pair in native FP64 (FP64 runs at 1/64 of the FP32 rate).
// ----------------------------------------------------------------------------
struct ff {
    float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)   // needs |a| >= |b| (or a == 0)
{
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sqr(ff a)
{
    const float p = __fmul_rn(a.h, a.h);
    float e = fmaf(a.h, a.h, -p);
    e = fmaf(__fadd_rn(a.h, a.h), a.l, e);
    return fast_two_sum(p, e);
}

// Split of an FP64 value into h + l (h = nearest float, l = nearest float to
// the exact remainder): 48 significant bits.
__host__ __device__ __forceinline__ void split_f64(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// Square root of a non-negative ff value: FP32 reciprocal square root
// refined by one FP32 Newton step, then one Newton correction in ff (about
// 2^-46 relative; the same steps as the eta of phi_ff_s).  0 for 0.
__device__ __forceinline__ ff ff_sqrt(ff s)
{
    const float sc = fmaxf(s.h, 1e-37f);
    float y = rsqrtf(sc);
    y = __fmul_rn(y, fmaf(-0.5f * sc, __fmul_rn(y, y), 1.5f));
    const float e0 = __fmul_rn(s.h, y);
    const float r = __fadd_rn(fmaf(-e0, e0, s.h), s.l);
    return fast_two_sum(e0, __fmul_rn(__fmul_rn(r, 0.5f), y));
}

// Bit pattern of a non-negative double: for such values the unsigned
// integer order is the numeric order, so maxima and comparisons of errors and
// bounds run on the integer pipe instead of the (slow) FP64 pipe.
__device__ __forceinline__ unsigned long long dbits(double x)
{
    return (unsigned long long)__double_as_longlong(x);
}

__device__ __forceinline__ double bitsd(unsigned long long b)
{
    return __longlong_as_double((long long)b);
}

// phi(eta) for s = eta^2 given as ff (coordinates pre-scaled by 1/R).
// sqrt: FP32 reciprocal square root refined by one Newton step in FP32, then
// one Newton correction of eta in ff (about 2^-46 relative).
__device__ __forceinline__ ff phi_ff_s(ff s)
{
    const float sc = fmaxf(s.h, 1e-37f);
    float y = rsqrtf(sc);
    y = __fmul_rn(y, fmaf(-0.5f * sc, __fmul_rn(y, y), 1.5f));
    const float e0 = __fmul_rn(s.h, y);
    const float r = __fadd_rn(fmaf(-e0, e0, s.h), s.l);
    const ff eta = fast_two_sum(e0, __fmul_rn(__fmul_rn(r, 0.5f), y));
    // 1 - eta.h by FastTwoSum (exact for eta.h <= 1; beyond, phi is set to 0)
    ff t = fast_two_sum(1.0f, -eta.h);
    t = fast_two_sum(t.h, __fsub_rn(t.l, eta.l));
    const ff t2 = ff_sqr(t);
    const ff t4 = ff_sqr(t2);
    ff p = two_sum(1.0f, __fmul_rn(4.0f, eta.h));
    p = fast_two_sum(p.h, __fmaf_rn(4.0f, eta.l, p.l));
    ff ph = ff_mul(t4, p);
    if (!(eta.h < 1.0f))
        ph = ff{0.0f, 0.0f};
    return ph;
}

// Squared scaled distance between an ff point and an ff centre.
__device__ __forceinline__ ff dist2_ff(float qxh, float qxl, float qyh, float qyl, float qzh,
                                       float qzl, float cxh, float cxl, float cyh, float cyl,
                                       float czh, float czl)
{
    ff dx = two_sum(qxh, -cxh);
    dx.l = __fadd_rn(dx.l, __fsub_rn(qxl, cxl));
    ff dy = two_sum(qyh, -cyh);
    dy.l = __fadd_rn(dy.l, __fsub_rn(qyl, cyl));
    ff dz = two_sum(qzh, -czh);
    dz.l = __fadd_rn(dz.l, __fsub_rn(qzl, czl));
    return ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
}

// ----------------------------------------------------------------------------
// Grid split of coordinates, for exact differences.  With 2^k above every
// |x| of a computation, G = 2^(k-23) and g = G 2^-24, a coordinate is stored
// as h = G rint(x / G) and l = g rint((x - h) / g): both are floats (at most
// 2^23 units of G or g), |x - h - l| <= g / 2 = 2^(k-48), and for two
// coordinates h1 - h2 and l1 - l2 are exact in FP32 (at most 2^24 units).
// The squared distance then needs no TwoSum on the differences.
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ double grid_unit(double xmax)
{
    int k = 0;
    frexp(xmax > 1e-30 ? xmax : 1e-30, &k);   // xmax = f 2^k, f in [0.5, 1)
    return ldexp(1.0, k - 23);
}

// Magnitude m (an integer) rounded to the nearest multiple of 2^sh, ties to
// even, returned as the count of 2^sh; sh >= 64 gives 0.
__host__ __device__ __forceinline__ uint64_t rne_shift(uint64_t m, int sh)
{
    if (sh <= 0)
        return m << (-sh);
    if (sh >= 64)
        return 0;
    const uint64_t q = m >> sh, rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

// The split with integer operations on the bits of x, which give exactly
// G rint(x / G) and g rint((x - h) / g) (ties to even): with |x| = M 2^E
// (M the 53-bit significand), H = M rounded at bit kg - E is the count of
// G, R = M - H 2^(kg - E) is x - h in units of 2^E (exact), and L = R
// rounded at bit kg - 24 - E is the count of g.  H and |L| are at most
// 2^23, so h = +-H G and l = +-L g are floats.  No FP64 arithmetic: FP64 is
// the slowest pipe of this GPU, and the rounding by FP64 divisions (or by
// adding and subtracting 1.5 2^52 G) made the packing of the volume points
// FP64-bound.  Zero and subnormal x (far below g) split into +0, +0, and a
// zero part is +0, as the FP64 rounding gives.
__host__ __device__ __forceinline__ void split_grid(double x, double G, float &h, float &l)
{
    uint64_t b, bg;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(x);
    bg = (uint64_t)__double_as_longlong(G);
#else
    memcpy(&b, &x, 8);
    memcpy(&bg, &G, 8);
#endif
    h = 0.0f;
    l = 0.0f;
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0)
        return;
    const int kg = (int)((bg >> 52) & 0x7ff) - 1023;            // G = 2^kg, kg >= -122
    const uint64_t M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const bool neg = (b >> 63) != 0;
    const int shH = kg - (e - 1075);                            // >= 30 when |x| < 2^(kg + 23)
    const uint64_t H = shH >= 54 ? 0 : rne_shift(M, shH);
    const int64_t R = shH >= 54 ? (int64_t)M : (int64_t)M - (int64_t)(H << shH);
    const bool rneg = R < 0;
    const uint64_t L = rne_shift(rneg ? (uint64_t)(-R) : (uint64_t)R, shH - 24);
#ifdef __CUDA_ARCH__
    const float Gf = __int_as_float((kg + 127) << 23);            // 2^kg, a normal float
#else
    const float Gf = ldexpf(1.0f, kg);
#endif
    const float gf = Gf * 5.9604644775390625e-08f;              // 2^(kg - 24), exact
    if (H)
        h = (neg ? -(float)(uint32_t)H : (float)(uint32_t)H) * Gf;
    if (L)
        l = ((neg != rneg) ? -(float)(uint32_t)L : (float)(uint32_t)L) * gf;
}

// Largest |x| / R over the volume points and the selected centres, as the
// bit pattern of a non-negative double (integer atomicMax keeps the order);
// it fixes the grid of the grid split (split_grid).
static __global__ void k_grid_max(const double *__restrict__ x, int64_t n, const double *__restrict__ xb,
                           const int32_t *__restrict__ sel, int64_t nc, double inv_r,
                           unsigned long long *__restrict__ out)
{
    // max |x| first, one scaling at the end: rounding is monotonic, so
    // fl(max |x| / R) = max fl(|x| / R)
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = fmax(mx, fabs(x[i]));
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nc;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = sel[j];
        mx = fmax(mx, fmax(fabs(xb[3 * q]), fmax(fabs(xb[3 * q + 1]), fabs(xb[3 * q + 2]))));
    }
    for (int o = 16; o > 0; o >>= 1)
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, (unsigned long long)__double_as_longlong(mx * inv_r));
}

__device__ __forceinline__ double grid_of(const unsigned long long *gmax)
{
    return grid_unit(__longlong_as_double((long long)*gmax));
}

// Squared distance of two grid-split points.  Per component the exact
// difference (qh - ch) + (ql - cl) is normalised by FastTwoSum (|qh - ch| is
// a multiple of G, so it is 0 or at least G >= |ql - cl|) and squared with an
// error-free product; the three squares are summed by two TwoSums, their low
// parts in FP32, and the result renormalised.
__device__ __forceinline__ void gs_square(float qh, float ql, float ch, float cl, float &p,
                                          float &e)
{
    const ff d = fast_two_sum(__fsub_rn(qh, ch), __fsub_rn(ql, cl));
    p = __fmul_rn(d.h, d.h);
    e = fmaf(d.h, d.h, -p);
    e = fmaf(__fadd_rn(d.h, d.h), d.l, e);
}

__device__ __forceinline__ ff dist2_gs(float qxh, float qxl, float qyh, float qyl, float qzh,
                                       float qzl, float cxh, float cxl, float cyh, float cyl,
                                       float czh, float czl)
{
    float px, ex, py, ey, pz, ez;
    gs_square(qxh, qxl, cxh, cxl, px, ex);
    gs_square(qyh, qyl, cyh, cyl, py, ey);
    gs_square(qzh, qzl, czh, czl, pz, ez);
    const ff s1 = two_sum(px, py);
    const ff s2 = two_sum(s1.h, pz);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), ez), __fadd_rn(s1.l, s2.l));
    return fast_two_sum(s2.h, lo);
}

// acc += w * phi with w and phi in ff; acc kept as an unnormalised pair whose
// low part collects the product and sum errors.
__device__ __forceinline__ void ff_fma_acc(ff &acc, float wh, float wl, ff ph)
{
    const float p = __fmul_rn(wh, ph.h);
    float pe = fmaf(wh, ph.h, -p);
    pe = fmaf(wh, ph.l, pe);
    pe = fmaf(wl, ph.h, pe);
    const ff s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, pe));
}

// ----------------------------------------------------------------------------
// Paired double-float: two independent ff values in paired FP32 registers, so
// every step of the error-free transformations serves two pairs with one
// instruction (same algorithms as above, lane by lane).
// ----------------------------------------------------------------------------
struct ff2 {
    f2 h, l;
};

__device__ __forceinline__ f2 f2_neg(f2 a)
{
    f2 r;
    r.v = a.v ^ 0x8000000080000000ull;
    return r;
}

__device__ __forceinline__ f2 f2_bcast(float x) { return f2_pack(x, x); }

__device__ __forceinline__ ff2 two_sum2(f2 a, f2 b)
{
    const f2 s = f2_add(a, b);
    const f2 bb = f2_sub(s, a);
    return ff2{s, f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}

__device__ __forceinline__ ff2 fast_two_sum2(f2 a, f2 b)
{
    const f2 s = f2_add(a, b);
    return ff2{s, f2_sub(b, f2_sub(s, a))};
}

// TwoSum of two non-negative paired values: FastTwoSum on (max, min) gives
// the same (s, e), since both compute the rounded sum and its exact error,
// with three FP32-pipe operations instead of six (and four min/max on the
// ALU pipe, which the pair kernels leave less busy).
__device__ __forceinline__ ff2 two_sum2_nn(f2 a, f2 b)
{
    float a0, a1, b0, b1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    return fast_two_sum2(f2_pack(fmaxf(a0, b0), fmaxf(a1, b1)),
                         f2_pack(fminf(a0, b0), fminf(a1, b1)));
}

__device__ __forceinline__ ff2 ff_add2(ff2 a, ff2 b)
{
    const ff2 s = two_sum2(a.h, b.h);
    return fast_two_sum2(s.h, f2_add(s.l, f2_add(a.l, b.l)));
}

__device__ __forceinline__ ff2 ff_mul2(ff2 a, ff2 b)
{
    const f2 p = f2_mul(a.h, b.h);
    f2 e = f2_fma(a.h, b.h, f2_neg(p));
    e = f2_fma(a.h, b.l, e);
    e = f2_fma(a.l, b.h, e);
    return fast_two_sum2(p, e);
}

__device__ __forceinline__ ff2 ff_sqr2(ff2 a)
{
    const f2 p = f2_mul(a.h, a.h);
    f2 e = f2_fma(a.h, a.h, f2_neg(p));
    e = f2_fma(f2_add(a.h, a.h), a.l, e);
    return fast_two_sum2(p, e);
}

// Squared scaled distances of two (query, centre) pairs given as paired
// hi/lo coordinates.
__device__ __forceinline__ ff2 dist2_ff2(f2 qxh, f2 qxl, f2 qyh, f2 qyl, f2 qzh, f2 qzl, f2 cxh,
                                         f2 cxl, f2 cyh, f2 cyl, f2 czh, f2 czl)
{
    ff2 dx = two_sum2(qxh, f2_neg(cxh));
    dx.l = f2_add(dx.l, f2_sub(qxl, cxl));
    ff2 dy = two_sum2(qyh, f2_neg(cyh));
    dy.l = f2_add(dy.l, f2_sub(qyl, cyl));
    ff2 dz = two_sum2(qzh, f2_neg(czh));
    dz.l = f2_add(dz.l, f2_sub(qzl, czl));
    return ff_add2(ff_add2(ff_sqr2(dx), ff_sqr2(dy)), ff_sqr2(dz));
}

// Squared distances of two (query, centre) pairs of grid-split points (the
// method of dist2_gs, lane by lane).
__device__ __forceinline__ void gs_square2(f2 qh, f2 ql, f2 ch, f2 cl, f2 &p, f2 &e)
{
    const ff2 d = fast_two_sum2(f2_sub(qh, ch), f2_sub(ql, cl));
    p = f2_mul(d.h, d.h);
    e = f2_fma(d.h, d.h, f2_neg(p));
    e = f2_fma(f2_add(d.h, d.h), d.l, e);
}

__device__ __forceinline__ ff2 dist2_gs2(f2 qxh, f2 qxl, f2 qyh, f2 qyl, f2 qzh, f2 qzl, f2 cxh,
                                         f2 cxl, f2 cyh, f2 cyl, f2 czh, f2 czl)
{
    f2 px, ex, py, ey, pz, ez;
    gs_square2(qxh, qxl, cxh, cxl, px, ex);
    gs_square2(qyh, qyl, cyh, cyl, py, ey);
    gs_square2(qzh, qzl, czh, czl, pz, ez);
    const ff2 s1 = two_sum2_nn(px, py);   // squares: non-negative
    const ff2 s2 = two_sum2_nn(s1.h, pz);
    const f2 lo = f2_add(f2_add(f2_add(ex, ey), ez), f2_add(s1.l, s2.l));
    return fast_two_sum2(s2.h, lo);
}

// phi for two pairs (same method as phi_ff_s; the reciprocal square roots
// are scalar MUFU operations).
__device__ __forceinline__ ff2 phi_ff2_s(ff2 s)
{
    float s0, s1;
    f2_unpack(s.h, s0, s1);
    const f2 sc = f2_pack(fmaxf(s0, 1e-37f), fmaxf(s1, 1e-37f));
    f2 y = f2_pack(rsqrtf(fmaxf(s0, 1e-37f)), rsqrtf(fmaxf(s1, 1e-37f)));
    y = f2_mul(y, f2_fma(f2_mul(f2_bcast(-0.5f), sc), f2_mul(y, y), f2_bcast(1.5f)));
    const f2 e0 = f2_mul(s.h, y);
    const f2 r = f2_add(f2_fma(f2_neg(e0), e0, s.h), s.l);
    const ff2 eta = fast_two_sum2(e0, f2_mul(f2_mul(r, f2_bcast(0.5f)), y));
    ff2 t = fast_two_sum2(f2_bcast(1.0f), f2_neg(eta.h));
    t = fast_two_sum2(t.h, f2_sub(t.l, eta.l));
    const ff2 t2 = ff_sqr2(t);
    const ff2 t4 = ff_sqr2(t2);
    ff2 p = two_sum2_nn(f2_bcast(1.0f), f2_mul(f2_bcast(4.0f), eta.h));   // eta >= 0
    p = fast_two_sum2(p.h, f2_fma(f2_bcast(4.0f), eta.l, p.l));
    ff2 ph = ff_mul2(t4, p);
    float e0a, e0b;
    f2_unpack(eta.h, e0a, e0b);
    float hh0, hh1, ll0, ll1;
    f2_unpack(ph.h, hh0, hh1);
    f2_unpack(ph.l, ll0, ll1);
    if (!(e0a < 1.0f)) {
        hh0 = 0.0f;
        ll0 = 0.0f;
    }
    if (!(e0b < 1.0f)) {
        hh1 = 0.0f;
        ll1 = 0.0f;
    }
    return ff2{f2_pack(hh0, hh1), f2_pack(ll0, ll1)};
}

// acc += w * phi for two pairs.
__device__ __forceinline__ void ff_fma_acc2(ff2 &acc, f2 wh, f2 wl, ff2 ph)
{
    const f2 p = f2_mul(wh, ph.h);
    f2 pe = f2_fma(wh, ph.h, f2_neg(p));
    pe = f2_fma(wh, ph.l, pe);
    pe = f2_fma(wl, ph.h, pe);
    const ff2 s = two_sum2(acc.h, p);
    acc.h = s.h;
    acc.l = f2_add(acc.l, f2_add(s.l, pe));
}

// ----------------------------------------------------------------------------
// Argmax keys: a container for an argmax candidate's node and the "no
// candidate" marker (key 0).
//  - The top 40 bits of the (non-negative) FP64 error's bit pattern, then 24
//    bits of (0xFFFFFF - node), so a key is never 0.  Candidates are ranked by
//    their exact error carried beside the key, then by the lower node index;
//    the truncated value in the key is not used for ranking.
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
// Bulk (TMA) copy global -> shared memory completed on an mbarrier.
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: expect `bytes` on the barrier and start the copy.  `bytes` and
// both addresses must be multiples of 16.  Global data written by other SMs
// (generic proxy) is ordered before the async-proxy read by the fence.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// One thread: one arrival that expects `bytes` in total from the copies
// started next with bulk_copy_g2s (fences as in bulk_g2s).
__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// A bulk copy whose bytes count against an expectation set by mbar_expect
// (no arrival of its own).  `bytes` and both addresses: multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for the barrier phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          uint64_t limit_ns)
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
        if (it == 0)
            t0 = globaltimer_ns();
        else if (globaltimer_ns() - t0 > limit_ns)
            return false;
    }
}

// ----------------------------------------------------------------------------
// Grid barrier for cooperative launches (all CTAs co-resident).  Flat,
// contention-free: CTA b publishes its arrival count in its own word with a
// release store (ordered after the CTA's writes by the preceding
// __syncthreads), and every CTA's warp 0 polls all the words with relaxed
// loads until each has reached the same count, then takes one acquire fence.
// No two CTAs write the same address, so an arrival costs one store instead
// of a serialised atomic, and the wait ends one L2 round trip after the last
// arrival.  Every wait is bounded: after `limit_ns` the waiting CTA latches
// RBF_E_TIMEOUT into *status and returns false; callers then leave the
// kernel.  The clock and the status word are read every 16th poll.
// ----------------------------------------------------------------------------
constexpr int kBarMaxCtas = 4096;

struct GridBar {
    unsigned int arrive[kBarMaxCtas];
};

// Time CTA 0 spent waiting in grid barriers (profiling), kept in shared
// memory: a global update after every barrier would delay CTA 0's next
// arrival.  A kernel that reports it zeroes it on entry.
static __shared__ unsigned long long g_bar_wait_ns;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// `epoch` counts the barriers this CTA has passed (the same in every CTA);
// `my_block` is the CTA's index among the nblocks taking part.
__device__ __forceinline__ bool grid_barrier(GridBar *bar, int *status, unsigned int nblocks,
                                             uint64_t limit_ns, unsigned int &epoch,
                                             unsigned int my_block)
{
    __shared__ int s_ok;
    const unsigned int target = epoch + 1;
    __syncthreads();
    if (threadIdx.x < 32) {
        int ok = 1;
        if (threadIdx.x == 0)
            st_release_u32(&bar->arrive[my_block], target);
        __syncwarp();
        const uint64_t t0 = globaltimer_ns();
        for (unsigned int poll = 1;; ++poll) {
            bool mine = true;
            for (unsigned int b = threadIdx.x; b < nblocks; b += 32)
                mine &= (int)(ld_relaxed_u32(&bar->arrive[b]) - target) >= 0;
            if (__all_sync(0xffffffffu, mine))
                break;
            if ((poll & 15u) == 0u) {
                if (*(volatile int *)status == (int)RBF_E_TIMEOUT) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > limit_ns) {
                    if (threadIdx.x == 0)
                        atomicExch(status, (int)RBF_E_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel_gpu();
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) {
            s_ok = ok;
            if (my_block == 0)
                g_bar_wait_ns += globaltimer_ns() - t0;
        }
    }
    __syncthreads();
    epoch = target;
    return s_ok != 0;
}

}  // namespace rbf
