// rbf_cull.cu -- volume displacement sum (Eq. 6) with compact-support culling.
//
// The Wendland C2 basis vanishes for eta = d / R >= 1 (Sec. 2), so a volume
// point receives nothing from centres farther than R.  A plan, made once per
// volume mesh and radius, sorts the points along a Morton (Z-order) curve of
// a uniform grid of cells and records the bounding box of every tile of
// consecutive sorted points (one CTA's points per step).  Each run then
// builds, per tile, the ordered list of centres whose distance to the tile's
// box is below R (with a margin) and sums only those pairs.
//
// A skipped centre is at least (1 + 1e-3) R from every point of the tile, so
// its pair would have been an exact zero: the FP32 kernel forces phi = 0 for
// eta^2 >= 1 and the double-float phi is zero there already.  The list keeps
// the centres in their original order, so every point's sum is the unculled
// sum with its zero terms left out: the result does not depend on the
// sort, the tiles or the order of points within a cell.
//
// Plan creation (all on the device): bounding box of the points, cell key of
// each point (b bits per axis, interleaved), a counting sort by key (warp-
// aggregated histogram, one-CTA exclusive scan, warp-aggregated scatter),
// the packed sorted coordinates (FP32, or double-float hi/lo) and the tile
// boxes.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kCullThreads = 256;
constexpr int kCullWarps = kCullThreads / kWarp;
constexpr int kCullP = 2;                                  // FP32: paired registers per thread
constexpr int kCullTileF32 = kCullThreads * 2 * kCullP;    // 1024 points per tile
constexpr int kCullQFF = 2;                                // double-float: points per thread
constexpr int kCullTileFF = kCullThreads * kCullQFF;       // 512 points per tile
constexpr int kCullChunkF32 = 2048;                        // centres per shared-memory chunk
constexpr int kCullChunkFF = 1024;
constexpr float kCullNear2 = 1.002001f;                    // (1 + 1e-3)^2: keep below
constexpr int kBboxBlocks = 1024;

// Dynamic shared memory of a run holding `cap` centres: the table and the
// list of near centres.
inline size_t cull_smem(bool ff, int cap)
{
    return sizeof(float4) * (ff ? 4 : 3) * (size_t)cap + sizeof(int) * (size_t)cap;
}

struct CullLayout {
    size_t box6, bpart, keys, cells, pts, pts_lo, perm, tbox, table, total;
    int bits, tile, chunk;
    int64_t ntiles, ncells;
};

static int cull_bits(int64_t nv)
{
    // about 8 points per cell, 3..7 bits per axis
    int b = 3;
    while (b < 7 && ((int64_t)1 << (3 * (b + 1))) * 8 <= nv)
        ++b;
    return b;
}

static CullLayout cull_layout(int64_t nv, int64_t nc_max, int prec)
{
    CullLayout L{};
    L.bits = cull_bits(nv);
    L.ncells = (int64_t)1 << (3 * L.bits);
    const bool ff = prec == RBF_PREC_F32X2;
    L.tile = ff ? kCullTileFF : kCullTileF32;
    L.chunk = ff ? kCullChunkFF : kCullChunkF32;
    L.ntiles = (nv + L.tile - 1) / L.tile;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.box6 = take(sizeof(double) * 8);
    L.bpart = take(sizeof(double) * 6 * kBboxBlocks);
    L.keys = take(sizeof(uint32_t) * (size_t)nv);
    L.cells = take(sizeof(uint32_t) * (size_t)L.ncells);
    L.pts = take(sizeof(float4) * (size_t)nv);
    L.pts_lo = take(ff ? sizeof(float4) * (size_t)nv : 0);
    L.perm = take(sizeof(int32_t) * (size_t)nv);
    L.tbox = take(sizeof(float4) * 2 * (size_t)L.ntiles);
    L.table = take(sizeof(float4) * (ff ? 4 : 3) * (size_t)std::max<int64_t>(nc_max, 1));
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// Plan creation kernels.
// ---------------------------------------------------------------------------
__global__ void k_cull_bbox_partial(const double *__restrict__ xv, int64_t nv, double inv_r,
                                    double *__restrict__ part)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const double v = xv[3 * i + c] * inv_r;
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    __shared__ double s[6][kCullWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
        if (lane == 0) {
            s[c][warp] = lo[c];
            s[3 + c][warp] = hi[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        double v = s[c][0];
        for (int w = 1; w < kCullWarps; ++w)
            v = c < 3 ? fmin(v, s[c][w]) : fmax(v, s[c][w]);
        part[6 * blockIdx.x + c] = v;
    }
}

__global__ void k_cull_bbox_final(const double *__restrict__ part, int nblk,
                                  double *__restrict__ box6)
{
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        double v = part[c];
        for (int b = 1; b < nblk; ++b)
            v = c < 3 ? fmin(v, part[6 * b + c]) : fmax(v, part[6 * b + c]);
        box6[c] = v;
    }
}

// Interleaves the low 10 bits of v with two zero bits between them (the
// usual magic-mask construction of a 3-D Morton code).
__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Cell key of every point and the per-cell counts (one atomic per group of
// lanes that share a key).
__global__ void k_cull_keys(const double *__restrict__ xv, int64_t nv, double inv_r,
                            const double *__restrict__ box6, int bits,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ cells)
{
    const double n = (double)(1u << bits);
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nv;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool act = i < nv;
        uint32_t key = 0xffffffffu;
        if (act) {
            uint32_t q[3];
            for (int c = 0; c < 3; ++c) {
                const double ext = box6[3 + c] - box6[c];
                const double u = ext > 0.0 ? (xv[3 * i + c] * inv_r - box6[c]) / ext : 0.0;
                q[c] = (uint32_t)fmin(fmax(u * n, 0.0), n - 1.0);
            }
            key = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
            keys[i] = key;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (act && lane == __ffs(peers) - 1)
            atomicAdd(cells + key, (uint32_t)__popc(peers));
    }
}

// Exclusive prefix sum of the cell counts, in place, by one CTA of 1024
// threads (each owns a contiguous run of cells).
__global__ void __launch_bounds__(1024) k_cull_scan(uint32_t *__restrict__ cells, int64_t n)
{
    __shared__ uint32_t s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (n + 1023) / 1024;
    const int64_t b0 = tid * per, b1 = min(n, b0 + per);
    uint32_t sum = 0;
    for (int64_t c = b0; c < b1; ++c)
        sum += cells[c];
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += v;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = s_w[lane], w = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += u;
        }
        s_w[lane] = w - v;   // exclusive over warps
    }
    __syncthreads();
    uint32_t run = s_w[warp] + incl - sum;
    for (int64_t c = b0; c < b1; ++c) {
        const uint32_t v = cells[c];
        cells[c] = run;
        run += v;
    }
}

// Counting-sort scatter: sorted position of every point, its original index
// and its packed scaled coordinates (FP32, or double-float hi and lo).
__global__ void k_cull_scatter(const double *__restrict__ xv, int64_t nv, double inv_r,
                               const uint32_t *__restrict__ keys, uint32_t *__restrict__ cursor,
                               int32_t *__restrict__ perm, float4 *__restrict__ pts,
                               float4 *__restrict__ pts_lo)
{
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nv;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool act = i < nv;
        const uint32_t key = act ? keys[i] : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t pos0 = 0;
        if (act && lane == leader)
            pos0 = atomicAdd(cursor + key, (uint32_t)__popc(peers));
        pos0 = __shfl_sync(0xffffffffu, pos0, leader);
        if (!act)
            continue;
        const uint32_t pos = pos0 + __popc(peers & ((1u << lane) - 1u));
        perm[pos] = (int32_t)i;
        const double x = xv[3 * i] * inv_r, y = xv[3 * i + 1] * inv_r, z = xv[3 * i + 2] * inv_r;
        if (pts_lo) {
            float h0, l0, h1, l1, h2, l2;
            split_f64(x, h0, l0);
            split_f64(y, h1, l1);
            split_f64(z, h2, l2);
            pts[pos] = make_float4(h0, h1, h2, 0.0f);
            pts_lo[pos] = make_float4(l0, l1, l2, 0.0f);
        } else {
            pts[pos] = make_float4((float)x, (float)y, (float)z, 0.0f);
        }
    }
}

// Box (lo, hi) of every tile of `tile` consecutive sorted points; one warp
// per tile.
__global__ void k_cull_tile_boxes(const float4 *__restrict__ pts, int64_t nv, int tile,
                                  int64_t ntiles, float4 *__restrict__ tbox)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = w0; t < ntiles; t += nw) {
        float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
        const int64_t p1 = min(nv, (t + 1) * (int64_t)tile);
        for (int64_t p = t * (int64_t)tile + lane; p < p1; p += 32) {
            const float4 v = pts[p];
            lo[0] = fminf(lo[0], v.x);
            lo[1] = fminf(lo[1], v.y);
            lo[2] = fminf(lo[2], v.z);
            hi[0] = fmaxf(hi[0], v.x);
            hi[1] = fmaxf(hi[1], v.y);
            hi[2] = fmaxf(hi[2], v.z);
        }
        for (int c = 0; c < 3; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
                hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
            }
        if (lane == 0) {
            tbox[2 * t] = make_float4(lo[0], lo[1], lo[2], 0.0f);
            tbox[2 * t + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
        }
    }
}

// ---------------------------------------------------------------------------
// Run kernels.
// ---------------------------------------------------------------------------
// Centre tables: FP32 (cx, cx, cy, cy), (cz, cz, wx, wx), (wy, wy, wz, wz)
// (duplicated for the paired registers); double-float (c_hi, c_lo, w_hi,
// w_lo).
__global__ void k_cull_pack_centres(const double *__restrict__ xb, const int32_t *__restrict__ sel,
                                    const double *__restrict__ w, int nc, double inv_r, int ff,
                                    float4 *__restrict__ tab)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        const int64_t n = sel[j];
        const double c[3] = {xb[3 * n] * inv_r, xb[3 * n + 1] * inv_r, xb[3 * n + 2] * inv_r};
        const double wv[3] = {w[3 * j], w[3 * j + 1], w[3 * j + 2]};
        if (ff) {
            float h[3], l[3], hw[3], lw[3];
            for (int k = 0; k < 3; ++k) {
                split_f64(c[k], h[k], l[k]);
                split_f64(wv[k], hw[k], lw[k]);
            }
            tab[4 * j] = make_float4(h[0], h[1], h[2], 0.0f);
            tab[4 * j + 1] = make_float4(l[0], l[1], l[2], 0.0f);
            tab[4 * j + 2] = make_float4(hw[0], hw[1], hw[2], 0.0f);
            tab[4 * j + 3] = make_float4(lw[0], lw[1], lw[2], 0.0f);
        } else {
            const float fx = (float)c[0], fy = (float)c[1], fz = (float)c[2];
            const float gx = (float)wv[0], gy = (float)wv[1], gz = (float)wv[2];
            tab[3 * j] = make_float4(fx, fx, fy, fy);
            tab[3 * j + 1] = make_float4(fz, fz, gx, gx);
            tab[3 * j + 2] = make_float4(gy, gy, gz, gz);
        }
    }
}

// Ordered list (in s_list) of the centres of the shared-memory chunk
// [0, nt) that lie within R (plus the margin) of the box [lo, hi]; `stride`
// float4 per centre, coordinates read by `cxyz`.  Returns the list length.
// All threads call it; it starts and ends with a barrier.
template <typename CXYZ>
__device__ __forceinline__ int build_near_list(int nt, float4 lo, float4 hi, int *s_list,
                                               int *s_wcnt, CXYZ cxyz)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int base = 0;
    __syncthreads();   // readers of the previous list are done
    for (int r0 = 0; r0 < nt; r0 += kCullThreads) {
        const int j = r0 + tid;
        bool near = false;
        if (j < nt) {
            float cx, cy, cz;
            cxyz(j, cx, cy, cz);
            const float dx = fmaxf(fmaxf(lo.x - cx, cx - hi.x), 0.0f);
            const float dy = fmaxf(fmaxf(lo.y - cy, cy - hi.y), 0.0f);
            const float dz = fmaxf(fmaxf(lo.z - cz, cz - hi.z), 0.0f);
            near = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < kCullNear2;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, near);
        if (lane == 0)
            s_wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = base, tot = 0;
        for (int w = 0; w < kCullWarps; ++w) {
            const int c = s_wcnt[w];
            off += w < warp ? c : 0;
            tot += c;
        }
        if (near)
            s_list[off + __popc(bal & ((1u << lane) - 1u))] = j;
        base += tot;
        __syncthreads();   // s_wcnt is rewritten by the next round
    }
    return base;
}

// phi of two squared distances with phi = 0 exactly where eta^2 >= 1.
__device__ __forceinline__ f2 phi_f32x2_cut(f2 s)
{
    float s0, s1, p0, p1;
    f2_unpack(s, s0, s1);
    f2_unpack(phi_f32x2_s(s), p0, p1);
    return f2_pack(s0 < 1.0f ? p0 : 0.0f, s1 < 1.0f ? p1 : 0.0f);
}

template <int P>
__global__ void __launch_bounds__(kCullThreads)
k_cull_volume_f32(const float4 *__restrict__ xs, const int32_t *__restrict__ perm, int64_t nv,
                  const float4 *__restrict__ tbox, const float4 *__restrict__ cw, int nc,
                  double *__restrict__ out, unsigned long long *__restrict__ pairs)
{
    extern __shared__ float4 s_cw[];
    const bool one_chunk = nc <= kCullChunkF32;
    int *s_list = (int *)(s_cw + 3 * (one_chunk ? nc : kCullChunkF32));
    __shared__ int s_wcnt[kCullWarps];
    const int tid = threadIdx.x;
    constexpr int T = kCullThreads * 2 * P;
    const int64_t ntiles = (nv + T - 1) / T;
    if (one_chunk) {
        for (int j = tid; j < 3 * nc; j += kCullThreads)
            s_cw[j] = cw[j];
    }
    auto cxyz = [&](int j, float &x, float &y, float &z) {
        const float4 A = s_cw[3 * j], B = s_cw[3 * j + 1];
        x = A.x;
        y = A.z;
        z = B.x;
    };
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * T;
        const float4 lo = tbox[2 * t], hi = tbox[2 * t + 1];
        f2 qx[P], qy[P], qz[P], ax[P], ay[P], az[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int64_t v0 = base + (int64_t)(2 * i) * kCullThreads + tid;
            int64_t v1 = v0 + kCullThreads;
            v0 = v0 < nv ? v0 : nv - 1;
            v1 = v1 < nv ? v1 : nv - 1;
            const float4 p0 = xs[v0], p1 = xs[v1];
            qx[i] = f2_pack(p0.x, p1.x);
            qy[i] = f2_pack(p0.y, p1.y);
            qz[i] = f2_pack(p0.z, p1.z);
            ax[i] = f2_pack(0.0f, 0.0f);
            ay[i] = ax[i];
            az[i] = ax[i];
        }
        unsigned long long visited = 0;
        for (int c0 = 0; c0 < nc; c0 += kCullChunkF32) {
            const int nt = min(kCullChunkF32, nc - c0);
            if (!one_chunk) {
                __syncthreads();
                for (int j = tid; j < 3 * nt; j += kCullThreads)
                    s_cw[j] = cw[3 * (size_t)c0 + j];
            }
            const int nl = build_near_list(nt, lo, hi, s_list, s_wcnt, cxyz);
            visited += (unsigned long long)nl;
#pragma unroll 2
            for (int k = 0; k < nl; ++k) {
                const int j = s_list[k];
                const float4 A = s_cw[3 * j], B = s_cw[3 * j + 1], C = s_cw[3 * j + 2];
                const f2 cx = f2_pack(A.x, A.y), cy = f2_pack(A.z, A.w), cz = f2_pack(B.x, B.y);
                const f2 wx = f2_pack(B.z, B.w), wy = f2_pack(C.x, C.y), wz = f2_pack(C.z, C.w);
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const f2 dx = f2_sub(qx[i], cx), dy = f2_sub(qy[i], cy), dz = f2_sub(qz[i], cz);
                    const f2 s = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                    const f2 ph = phi_f32x2_cut(s);
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
            const int64_t v0 = base + (int64_t)(2 * i) * kCullThreads + tid;
            const int64_t v1 = v0 + kCullThreads;
            if (v0 < nv) {
                const int64_t o = perm[v0];
                out[3 * o] = (double)x0;
                out[3 * o + 1] = (double)y0;
                out[3 * o + 2] = (double)z0;
            }
            if (v1 < nv) {
                const int64_t o = perm[v1];
                out[3 * o] = (double)x1;
                out[3 * o + 1] = (double)y1;
                out[3 * o + 2] = (double)z1;
            }
        }
        if (tid == 0 && pairs && visited)
            atomicAdd(pairs, visited * (unsigned long long)(int64_t)min((long long)T, (long long)(nv - base)));
    }
}

template <int Q>
__global__ void __launch_bounds__(kCullThreads)
k_cull_volume_ff(const float4 *__restrict__ xh, const float4 *__restrict__ xl,
                 const int32_t *__restrict__ perm, int64_t nv, const float4 *__restrict__ tbox,
                 const float4 *__restrict__ cw, int nc, double *__restrict__ out,
                 unsigned long long *__restrict__ pairs)
{
    static_assert(Q % 2 == 0, "points per thread come in pairs");
    constexpr int P = Q / 2;
    extern __shared__ float4 s_cwff[];
    const bool one_chunk = nc <= kCullChunkFF;
    int *s_list = (int *)(s_cwff + 4 * (one_chunk ? nc : kCullChunkFF));
    __shared__ int s_wcnt[kCullWarps];
    const int tid = threadIdx.x;
    constexpr int T = kCullThreads * Q;
    const int64_t ntiles = (nv + T - 1) / T;
    if (one_chunk) {
        for (int j = tid; j < 4 * nc; j += kCullThreads)
            s_cwff[j] = cw[j];
    }
    auto cxyz = [&](int j, float &x, float &y, float &z) {
        const float4 A = s_cwff[4 * j];
        x = A.x;
        y = A.y;
        z = A.z;
    };
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * T;
        const float4 lo = tbox[2 * t], hi = tbox[2 * t + 1];
        f2 qxh[P], qxl[P], qyh[P], qyl[P], qzh[P], qzl[P];
        ff2 ax[P], ay[P], az[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int64_t v0 = base + (int64_t)(2 * i) * kCullThreads + tid;
            int64_t v1 = v0 + kCullThreads;
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
        unsigned long long visited = 0;
        for (int c0 = 0; c0 < nc; c0 += kCullChunkFF) {
            const int nt = min(kCullChunkFF, nc - c0);
            if (!one_chunk) {
                __syncthreads();
                for (int j = tid; j < 4 * nt; j += kCullThreads)
                    s_cwff[j] = cw[4 * (size_t)c0 + j];
            }
            const int nl = build_near_list(nt, lo, hi, s_list, s_wcnt, cxyz);
            visited += (unsigned long long)nl;
            for (int k = 0; k < nl; ++k) {
                const int j = s_list[k];
                const float4 ch = s_cwff[4 * j], cl = s_cwff[4 * j + 1];
                const float4 wh = s_cwff[4 * j + 2], wl = s_cwff[4 * j + 3];
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const ff2 s2 = dist2_ff2(qxh[i], qxl[i], qyh[i], qyl[i], qzh[i], qzl[i],
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
            const int64_t v0 = base + (int64_t)(2 * i) * kCullThreads + tid;
            const int64_t v1 = v0 + kCullThreads;
            if (v0 < nv) {
                const int64_t o = perm[v0];
                out[3 * o] = (double)xh0 + (double)xl0;
                out[3 * o + 1] = (double)yh0 + (double)yl0;
                out[3 * o + 2] = (double)zh0 + (double)zl0;
            }
            if (v1 < nv) {
                const int64_t o = perm[v1];
                out[3 * o] = (double)xh1 + (double)xl1;
                out[3 * o + 1] = (double)yh1 + (double)yl1;
                out[3 * o + 2] = (double)zh1 + (double)zl1;
            }
        }
        if (tid == 0 && pairs && visited)
            atomicAdd(pairs, visited * (unsigned long long)(int64_t)min((long long)T, (long long)(nv - base)));
    }
}

}  // namespace rbf

using namespace rbf;

struct rbf_volume_plan {
    CullLayout L;
    char *ws;
    int64_t nv;
    int64_t nc_max;
    double radius;
    int prec;
    int sms;
};

extern "C" size_t rbf_volume_plan_workspace_bytes(int64_t nv, const rbf_params *p)
{
    if (!p || nv < 1 || nv > INT32_MAX || p->nc_max < 1 ||
        (p->eval_prec != RBF_PREC_F32 && p->eval_prec != RBF_PREC_F32X2))
        return 0;
    return cull_layout(nv, p->nc_max, p->eval_prec).total;
}

extern "C" rbf_status rbf_volume_plan_create(const double *d_xv, int64_t nv, const rbf_params *p,
                                             void *d_ws, size_t ws_bytes, void *stream,
                                             rbf_volume_plan **out)
{
    if (!out)
        return RBF_E_ARG;
    *out = nullptr;
    if (!p || !d_xv || nv < 1 || nv > INT32_MAX || p->nc_max < 1 || p->nc_max > (1 << 30) ||
        !(p->radius > 0.0) || (p->eval_prec != RBF_PREC_F32 && p->eval_prec != RBF_PREC_F32X2))
        return RBF_E_ARG;
    const CullLayout L = cull_layout(nv, p->nc_max, p->eval_prec);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    const double inv_r = 1.0 / p->radius;
    const bool ff = p->eval_prec == RBF_PREC_F32X2;
    double *box6 = (double *)(ws + L.box6);
    double *bpart = (double *)(ws + L.bpart);
    uint32_t *keys = (uint32_t *)(ws + L.keys), *cells = (uint32_t *)(ws + L.cells);
    float4 *pts = (float4 *)(ws + L.pts), *pts_lo = ff ? (float4 *)(ws + L.pts_lo) : nullptr;
    int32_t *perm = (int32_t *)(ws + L.perm);
    float4 *tbox = (float4 *)(ws + L.tbox);
    const int nblk = (int)std::min<int64_t>((nv + 255) / 256, kBboxBlocks);
    k_cull_bbox_partial<<<nblk, kCullThreads, 0, st>>>(d_xv, nv, inv_r, bpart);
    k_cull_bbox_final<<<1, 32, 0, st>>>(bpart, nblk, box6);
    if (cudaMemsetAsync(cells, 0, sizeof(uint32_t) * (size_t)L.ncells, st) != cudaSuccess)
        return RBF_E_CUDA;
    const int gb = (int)std::min<int64_t>((nv + 255) / 256, (int64_t)dev.sms * 8);
    k_cull_keys<<<gb, 256, 0, st>>>(d_xv, nv, inv_r, box6, L.bits, keys, cells);
    k_cull_scan<<<1, 1024, 0, st>>>(cells, L.ncells);
    k_cull_scatter<<<gb, 256, 0, st>>>(d_xv, nv, inv_r, keys, cells, perm, pts, pts_lo);
    const int tb = (int)std::min<int64_t>((L.ntiles * 32 + 255) / 256, (int64_t)dev.sms * 8);
    k_cull_tile_boxes<<<tb, 256, 0, st>>>(pts, nv, L.tile, L.ntiles, tbox);
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    // largest shared memory of a run: a full centre chunk and its list
    const cudaError_t ea = ff ? cudaFuncSetAttribute(k_cull_volume_ff<kCullQFF>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)cull_smem(true, kCullChunkFF))
                              : cudaFuncSetAttribute(k_cull_volume_f32<kCullP>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)cull_smem(false, kCullChunkF32));
    if (ea != cudaSuccess)
        return RBF_E_CUDA;
    rbf_volume_plan *pl = new rbf_volume_plan();
    pl->L = L;
    pl->ws = ws;
    pl->nv = nv;
    pl->nc_max = p->nc_max;
    pl->radius = p->radius;
    pl->prec = p->eval_prec;
    pl->sms = dev.sms;
    *out = pl;
    return RBF_OK;
}

extern "C" rbf_status rbf_volume_plan_run(const rbf_volume_plan *pl, const double *d_xb,
                                          const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                                          double *d_dv, unsigned long long *d_pairs, void *stream)
{
    if (!pl || !d_dv || nc < 0 || nc > pl->nc_max || (nc > 0 && (!d_xb || !d_sel_idx || !d_w)))
        return RBF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (nc == 0)
        return cudaMemsetAsync(d_dv, 0, sizeof(double) * 3 * (size_t)pl->nv, st) == cudaSuccess
                   ? RBF_OK
                   : RBF_E_CUDA;
    const CullLayout &L = pl->L;
    char *ws = pl->ws;
    const bool ff = pl->prec == RBF_PREC_F32X2;
    float4 *tab = (float4 *)(ws + L.table);
    const int cb = (int)std::min<int64_t>((nc + 255) / 256, 1024);
    k_cull_pack_centres<<<cb, 256, 0, st>>>(d_xb, d_sel_idx, d_w, (int)nc, 1.0 / pl->radius,
                                            ff ? 1 : 0, tab);
    const float4 *pts = (const float4 *)(ws + L.pts);
    const int32_t *perm = (const int32_t *)(ws + L.perm);
    const float4 *tbox = (const float4 *)(ws + L.tbox);
    // resident CTAs per SM for this launch's shared memory
    const size_t smem = cull_smem(ff, (int)std::min<int64_t>(nc, ff ? kCullChunkFF : kCullChunkF32));
    int occ = 1;
    const cudaError_t eo =
        ff ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cull_volume_ff<kCullQFF>,
                                                           kCullThreads, smem)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cull_volume_f32<kCullP>,
                                                           kCullThreads, smem);
    if (eo != cudaSuccess)
        return RBF_E_CUDA;
    const int grid = (int)std::min<int64_t>(L.ntiles, (int64_t)pl->sms * std::max(occ, 1));
    if (ff)
        k_cull_volume_ff<kCullQFF><<<grid, kCullThreads, smem, st>>>(
            pts, (const float4 *)(ws + L.pts_lo), perm, pl->nv, tbox, tab, (int)nc, d_dv, d_pairs);
    else
        k_cull_volume_f32<kCullP><<<grid, kCullThreads, smem, st>>>(pts, perm, pl->nv, tbox, tab,
                                                                    (int)nc, d_dv, d_pairs);
    return cudaGetLastError() == cudaSuccess ? RBF_OK : RBF_E_CUDA;
}

extern "C" rbf_status rbf_volume_plan_info(const rbf_volume_plan *pl, int *bits_per_axis,
                                           int64_t *points_per_tile, int64_t *tiles)
{
    if (!pl)
        return RBF_E_ARG;
    if (bits_per_axis)
        *bits_per_axis = pl->L.bits;
    if (points_per_tile)
        *points_per_tile = pl->L.tile;
    if (tiles)
        *tiles = pl->L.ntiles;
    return RBF_OK;
}

extern "C" void rbf_volume_plan_destroy(rbf_volume_plan *pl) { delete pl; }
