// rbf_greedy.cu -- persistent GCB greedy selection of support nodes
// (Algorithm 1 of arXiv:2004.04817; m = 1 is the plain Rendall-Allen greedy).
//
// One cooperative launch runs the whole loop on the device:
//   prologue : pack the boundary nodes in group order (groups contiguous),
//              E* = tol * max |dr| if relative, three seed nodes, append them;
//   iteration: errors E_q in the active group G_(k mod m) (FP64, or FP32 /
//              double-float with an error bound, certified from the bounds or
//              by an FP64 re-score of every node whose bound reaches the
//              leader's), grid argmax (lowest node on ties), append when
//              E > E*; the run stops after m consecutive iterations without an
//              append (they visited every node with one set of weights), and
//              idle runs are shortened by look-ahead scans that certify the
//              iterations before the next group able to append.
// The Cholesky factor of Phi_SS grows by one row per appended node (the
// recurrence Cholesky of Sec. 1).  The kernel keeps Z = L^-1 (and Z^T) in
// FP64, so an append is two matrix-vector products (l = Z b, u = Z^T l) that
// spread over the whole grid, instead of a triangular solve whose k-step
// dependency chain would run on one SM:
//   l = Z b,  d = sqrt(1 - l.l),  y_new = (dr_n - l.y) / d,
//   new row of Z = [-u^T / d, 1 / d],  W <- W - u y_new / d,  w_new = y_new / d.
// Grid barriers are bounded (RBF_E_TIMEOUT instead of a hang).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

// Index of this CTA among the CTAs that run one problem, and their number.
// A single-problem launch uses the hardware ids; a batched launch gives each
// problem a contiguous range of CTAs.  Set by each kernel on entry.
__shared__ int g_vb;
__shared__ int g_vg;
// The grid barrier in use: the control block's own, or the candidate that
// the greedy's start-up calibration found fastest.
__shared__ GridBar *g_bar;

constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / kWarp;
constexpr int kMaxGrid = 4096;
constexpr int kBarCand = 8;            // candidate barrier locations
constexpr int kBarCandWords = 1088;    // flags per candidate (4,352-byte stride)
constexpr int kBarCalRounds = 4;       // timed barriers per candidate
constexpr int kBarCalMinCtas = 8;      // smaller grids keep the control block's barrier
constexpr int kSmemCentresF32 = 2048;      // FP32 centres staged in shared memory by the
constexpr int kSmemCentresFF = 1024;       // batched launch (64 KB, two CTAs per SM); the
                                           // single-problem launch (one CTA per SM) stages
                                           // up to the device's shared-memory limit
constexpr double kPivotMin = 1e-13;        // d^2 at or below: singular (coincident nodes)
constexpr int kLookIdle = 8;               // idle iterations before a look-ahead
constexpr int kLookChunk = 16;             // groups per look-ahead evaluation
// Pairs one CTA evaluates in about the time of one idle iteration (measured
// on the 50,000-node wing: 0.76 G double-float pairs/s per CTA, ~13 us per
// iteration), by precision; a look-ahead runs only when scanning one group
// costs at most half an idle iteration (see the main loop).
constexpr double kLookPairsFF = 8000.0, kLookPairsF32 = 40000.0, kLookPairsF64 = 400.0;
constexpr float kU32 = 5.9604645e-8f;      // u = 2^-24, unit roundoff of FP32
constexpr float kU32Sq = 3.5527137e-15f;   // u^2 = 2^-48, the double-float error unit
constexpr int kFFRenorm = 8;               // double-float accumulators renormalised every
                                           // kFFRenorm terms (bounds the low-part growth)
// Certified error bounds of the screened evaluation.  For a node q with
// sums over nc centres split over a team of ts lanes (n_l = ceil(nc / ts)
// terms per lane, log2(ts) levels of the team sum), X = max |x / R| over the
// boundary, W1 = sum_j |w_j|_1, sb = sum_j |w_j|_1 phi_qj (both as computed),
// |dr|_1 and the computed error E~, the derivation (phi Lipschitz with
// constant 2.109375 and |phi'(eta) eta| <= 0.6912 on [0, 1]; sqrt.approx.f32
// and rsqrtf within 2^-22 relative, which rbf_measure_approx_error checks)
// gives, with u = 2^-24:
//   FP32:         |E~ - E| <= u   ((n_l + log2 ts + 10) sb + |dr|_1
//                                  + (7.32 X + 4.5) W1 + 4.24 E~)
//   double-float: |E~ - E| <= u^2 ((9.5 n_ch + 3 log2 ts + 43) sb + 4 |dr|_1
//                                  + (14.7 X + 44) W1 + 50 E~)
// (n_ch = ceil(n_l / 2) + 1 terms per accumulator chain, renormalised every
// kFFRenorm terms; chains of more than 16 terms are summed in blocks of
// kFFRenorm, with 3 ceil(n_ch / 8) + 114 in place of 9.5 n_ch + 43), each
// times 1 + (2 n_l + 2 log2 ts + nc / 32 + 40) u for
// the second-order terms, the FP32 sums sb and W1 and the FP32 evaluation of
// the bound itself.  E is the exact error of q with the weights as held in
// the evaluation table.

struct GreedyCtl {
    GridBar bar;
    int status;
    int pad0;
    unsigned long long tslot[3];  // screen thresholds (bits of a non-negative double, ring)
    double estar;
    long long nc;
    long long iterations;
    long long full_checks;
    long long pairs_f32;
    long long pairs_f64;
    long long pairs_ff;
    unsigned long long rescored;
    double final_max;
    double final_rms;
    double min_pivot;
    double max_resid;
    long long n_hist;
    unsigned long long phase_ns[12];  // CTA 0's time per phase (see rbf_greedy_stats)
    long long barriers;               // grid barriers passed
    // Candidate locations of the grid barrier's flags.  How long a barrier
    // takes depends on where its flags live (the same launch measured 1.1
    // and 2.6 us per barrier at workspace offsets a few KB apart), so the
    // greedy times a few barriers on each candidate and keeps the fastest.
    // The stride (4 KB + 256 B) varies the address bits above the line.
    int bar_pick;
    int pad1;
    unsigned int bar_cand[kBarCand][kBarCandWords];
};
// The host reads back the statistics only (everything before the candidates).
constexpr size_t kCtlStatBytes = offsetof(GreedyCtl, bar_pick);

// Per-CTA record of an evaluation (see evaluate).
// mx, u1, u2: bit patterns of non-negative doubles (0 = none); sq: FP32.
struct __align__(16) EvalRec {
    unsigned long long mx, u1, u2;
    double e_lead, b_lead;
    float sq;
    int pad;
    long long n1, key, p_lead;
    long long first;   // look-ahead: smallest cyclic rank of a node above E*
};
constexpr long long kNoRank = 0x7FFFFFFFFFFFFFFFll;
static_assert(sizeof(EvalRec) == 80, "EvalRec is read as five 16-byte vectors");
__device__ constexpr EvalRec kEmptyRec{0, 0, 0, 0.0, 0.0, 0.0f, 0, -1, 0, -1, kNoRank};

struct GreedyArgs {
    const double *xb;
    const double *db;
    int nb;
    int m;
    int nc_max;
    int prec;
    double inv_r;
    double tol;
    int tol_mode;
    int flags;
    unsigned long long barrier_ns;   // bound of every grid-barrier wait
    int ld;                       // leading dimension of Z, Z^T (= nc_max)
    int32_t *sel_idx;
    int64_t *sel_iter;
    double *hist;
    int64_t hist_cap;
    GreedyCtl *ctl;
    const int32_t *perm;
    int32_t *node_of_pos;
    int32_t *pos_of_node;
    D4 *xg64;                // scaled coordinates, group order
    D4 *dg64;                // displacements, group order
    float4 *xg32;                 // FP32 coordinates = high parts of the double-float split
    float4 *xgl;                  // low parts (x/R - xg32), group order
    float4 *dgh, *dgl;            // displacements as double-float (high, low), group order
    uint8_t *in_s;
    float *u32;                   // FP32 upper bound of E per position
    double *e64;                  // FP64 E per position (last evaluation)
    double *part;                 // 2 x kMaxGrid x 4 reduction partials
    long long *parti;             // 2 x kMaxGrid index partials
    int32_t *spos;                // support positions
    D4 *c64;                 // support centres (scaled)
    D4 *w64;                 // weights
    float4 *cw32;                 // FP32 table, 2 planes of ld float4: centres, weights
    float4 *cwff;                 // double-float table, 4 planes of ld float4: centre hi,
                                  // centre lo, weight hi, weight lo (planes, so that the
                                  // lanes of a team read consecutive 16-byte entries)
    D4 *y64;                 // forward-solve vector y = Z dr_S
    double *z;                    // Z = L^-1, row-major, ld
    double *zt;                   // Z^T, row-major, ld
    double *bvec;
    double *lvec;
    EvalRec *rec;                 // 2 x kMaxGrid evaluation records
    D4 *rvec;                     // refinement residual / correction vectors
    D4 *tvec;
    double *w_out;                // optional FP64 weights output (nc x 3)
    int refine_steps;
    long long *nc_out;            // optional: |S| at exit (device, for batched runs)
    int smem_cap;                 // centres whose evaluation table fits in the launch's
                                  // dynamic shared memory (larger sets are read from L2)
    int peaks;                    // peak selection: nodes appended per iteration (<= 1: Alg. 1)
    double sep2;                  // and their squared separation, in units of R
    double *bmat;                 // block append: B = Phi(S, new), ld x 16, row-major
    double *lmat;                 // Lambda = Z B, ld x 16
    double *cmat;                 // Phi(new, new), 16 x 16
    double *bpart;                // per-CTA partial sums (kPeakGrid x kBlkV)
};

constexpr int kMaxPeaks = 16;
// groups of up to this many positions are selected by every CTA on its own
// (no grid barrier); larger groups are split over the grid, one record
// exchange per round
constexpr int kPeakBlockPositions = 2048;
// block append of up to kMaxPeaks nodes: per-CTA partial sums (the K' x K'
// Gram matrix of Lambda and Lambda^T y, K' = K rounded up to a power of two)
// and the largest grid of the peak-selection launch
constexpr int kBlkV = kMaxPeaks * kMaxPeaks + 3 * kMaxPeaks;
constexpr int kBlkSeg = 8;   // CTA segments of the grid sums
constexpr int kPeakGrid = 256;

// One candidate of a selection round, and the merge of two: the largest
// stored error (lowest node on ties) and, for the certification, the two
// largest upper bounds E~ + beta (as FP32 rounded up).
struct PeakCand {
    unsigned long long eb;   // bits of the stored error (non-negative double)
    unsigned int u1, u2;     // bits of the largest / second largest upper bound
    int node, pos, n1;       // winner's node and position (-1: none); node of u1
    float beta;              // winner's bound
};

__device__ __forceinline__ PeakCand peak_empty()
{
    return PeakCand{0ull, 0u, 0u, -1, -1, -1, 0.0f};
}

__device__ __forceinline__ void peak_merge(PeakCand &A, const PeakCand &B)
{
    if (B.pos >= 0 && (A.pos < 0 || B.eb > A.eb || (B.eb == A.eb && B.node < A.node))) {
        A.eb = B.eb;
        A.node = B.node;
        A.pos = B.pos;
        A.beta = B.beta;
    }
    if (B.n1 >= 0 && (A.n1 < 0 || B.u1 > A.u1 || (B.u1 == A.u1 && B.n1 < A.n1))) {
        A.u2 = max(A.u1, B.u2);
        A.u1 = B.u1;
        A.n1 = B.n1;
    } else {
        A.u2 = max(A.u2, B.u1);
    }
}

__device__ __forceinline__ void peak_warp_reduce(PeakCand &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PeakCand t;
        t.eb = __shfl_xor_sync(0xffffffffu, c.eb, o);
        t.u1 = __shfl_xor_sync(0xffffffffu, c.u1, o);
        t.u2 = __shfl_xor_sync(0xffffffffu, c.u2, o);
        t.node = __shfl_xor_sync(0xffffffffu, c.node, o);
        t.pos = __shfl_xor_sync(0xffffffffu, c.pos, o);
        t.n1 = __shfl_xor_sync(0xffffffffu, c.n1, o);
        t.beta = __shfl_xor_sync(0xffffffffu, c.beta, o);
        peak_merge(c, t);
    }
}

// |x_q - x_p|^2 < sep2 (scaled coordinates) for position q and a node taken
// earlier.  Screened in FP32 from the double-float split (relative error of
// the squared distance below 5e-7, against a margin of 4e-6 sep2 plus
// 1e-12 X^2); decided in FP64 near the boundary, so the answer is the FP64
// one.
__device__ __forceinline__ bool peak_too_close(const GreedyArgs &a, int q, const float4 &qh,
                                               const float4 &ql, const float4 &ph,
                                               const float4 &pl, const D4 &px, float s2f,
                                               float marg)
{
    const float dx = (qh.x - ph.x) + (ql.x - pl.x), dy = (qh.y - ph.y) + (ql.y - pl.y),
                dz = (qh.z - ph.z) + (ql.z - pl.z);
    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (d2 < s2f - marg)
        return true;
    if (d2 > s2f + marg)
        return false;
    const D4 x = ldcg(a.xg64 + q);
    const double ex = x.x - px.x, ey = x.y - px.y, ez = x.z - px.z;
    return fma(ez, ez, fma(ey, ey, ex * ex)) < a.sep2;
}

// Peak selection in the positions [p0, p1), called by every thread of every
// CTA: up to a.peaks nodes outside S with E > E*, in decreasing error (lowest
// node on ties), each at least sqrt(a.sep2) R from the nodes taken before it
// in this call.  The stored errors are E~ with bounds u32 (0 once re-scored
// in FP64).  With `exact` (FP64 values for every candidate) the stored
// errors decide directly; otherwise a round counts only when the bounds
// certify it (the winner's lower bound E~ - beta exceeds E* and every other
// eligible node's upper bound) and the call returns -1 at the first round
// they do not.  Returns -2 when a grid barrier gave up.
//
// One round is one pass over the positions: every thread keeps a bit per
// position it owns for "not a candidate any more" (in S, E <= E*, or too
// close to or equal to a node taken in an earlier round), so a later round
// tests only the newest node.  Small groups: every CTA scans the whole group and
// reaches the same choice without a barrier; large groups: each CTA scans a
// slice and the CTAs' candidates meet in one record exchange per round.
__device__ __forceinline__ int select_peaks(const GreedyArgs &a, int p0, int p1, double estar,
                                         bool exact, float xscale, int &use,
                                         unsigned int &epoch, int *pk_pos, int *pk_node,
                                         D4 *pk_x, float4 *pk_h, float4 *pk_l)
{
    __shared__ PeakCand s_pc[kGWarps];
    __shared__ PeakCand s_win;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = g_vg;
    const bool gmode = p1 - p0 > kPeakBlockPositions;
    const int base = gmode ? g_vb * kGThreads + tid : tid;
    const int stride = gmode ? G * kGThreads : kGThreads;
    const int K = min(a.peaks, kMaxPeaks);
    const unsigned long long es_bits = dbits(estar);
    const float es_dn = __double2float_rd(estar);
    const float s2f = (float)a.sep2;
    const float marg = 4e-6f * s2f + 1e-12f * xscale * xscale;
    unsigned int out = 0u;   // bit j: the thread's j-th position is no candidate
    int cnt = 0;
    for (int r = 0; r < K; ++r) {
        PeakCand c = peak_empty();
        int j = 0;
        for (int q = p0 + base; q < p1; q += stride, ++j) {
            const bool tracked = j < 32;
            if (tracked && ((out >> j) & 1u))
                continue;
            bool drop = false;
            const double e = ldcg(a.e64 + q);
            const float beta = exact ? 0.0f : ldcg(a.u32 + q);
            float up = 0.0f;
            if (r == 0 || !tracked) {
                if (ldcg(a.in_s + q)) {
                    drop = true;
                } else if (exact) {
                    drop = !(dbits(e) > es_bits);
                } else {
                    up = __fadd_ru(__double2float_ru(e), beta);
                    if (!(dbits(e) > es_bits))
                        drop = beta == 0.0f || up <= es_dn || !(e + (double)beta > estar);
                }
            } else if (!exact) {
                up = __fadd_ru(__double2float_ru(e), beta);
            }
            if (!drop && cnt > 0) {
                const float4 qh = ldcg(a.xg32 + q), ql = ldcg(a.xgl + q);
                const int u0 = tracked ? cnt - 1 : 0;
                for (int u = u0; u < cnt && !drop; ++u)
                    drop = q == pk_pos[u] ||
                           peak_too_close(a, q, qh, ql, pk_h[u], pk_l[u], pk_x[u], s2f, marg);
            }
            if (drop) {
                if (tracked)
                    out |= 1u << j;
                continue;
            }
            PeakCand t;
            t.eb = dbits(e);
            t.node = ldcg(a.node_of_pos + q);
            t.pos = q;
            t.beta = beta;
            t.u1 = __float_as_uint(up);
            t.u2 = 0u;
            t.n1 = exact ? -1 : t.node;
            peak_merge(c, t);
        }
        peak_warp_reduce(c);
        if (lane == 0)
            s_pc[warp] = c;
        __syncthreads();
        if (warp == 0) {
            PeakCand t = lane < kGWarps ? s_pc[lane] : peak_empty();
            peak_warp_reduce(t);
            if (lane == 0) {
                if (gmode)
                    ((PeakCand *)(a.rec + (size_t)(use & 1) * kMaxGrid))[g_vb] = t;
                else
                    s_win = t;
            }
        }
        if (gmode) {
            if (!grid_barrier(g_bar, &a.ctl->status, (unsigned)G, a.barrier_ns, epoch,
                              (unsigned)g_vb))
                return -2;
            if (warp == 0) {
                const PeakCand *rb = (const PeakCand *)(a.rec + (size_t)(use & 1) * kMaxGrid);
                PeakCand t = peak_empty();
                for (int b = lane; b < G; b += 32) {
                    PeakCand o;
                    o.eb = __ldcg(&rb[b].eb);
                    o.u1 = __ldcg(&rb[b].u1);
                    o.u2 = __ldcg(&rb[b].u2);
                    o.node = __ldcg(&rb[b].node);
                    o.pos = __ldcg(&rb[b].pos);
                    o.n1 = __ldcg(&rb[b].n1);
                    o.beta = __ldcg(&rb[b].beta);
                    peak_merge(t, o);
                }
                peak_warp_reduce(t);
                if (lane == 0)
                    s_win = t;
            }
            ++use;
        }
        __syncthreads();
        const PeakCand w = s_win;
        if (w.pos < 0)
            break;   // no candidate left
        if (!exact) {
            const double lower = bitsd(w.eb) - (double)w.beta;
            const float up = __uint_as_float(w.n1 != w.node ? w.u1 : w.u2);
            if (!(lower > estar) || !(lower > (double)up))
                return -1;
        }
        if (tid == 0) {
            pk_pos[cnt] = w.pos;
            pk_node[cnt] = w.node;
            pk_x[cnt] = ldcg(a.xg64 + w.pos);
            pk_h[cnt] = ldcg(a.xg32 + w.pos);
            pk_l[cnt] = ldcg(a.xgl + w.pos);
        }
        __syncthreads();
        ++cnt;
    }
    return cnt;
}

__device__ __forceinline__ int goff(int i, int nb, int m)
{
    const int base = nb / m, rem = nb % m;
    return i * base + min(i, rem);
}

// (value, index) pair reductions: larger value wins, lowest index on ties.
__device__ __forceinline__ void pick(double &v, long long &i, double v2, long long i2)
{
    if (v2 > v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i))) {
        v = v2;
        i = i2;
    }
}

struct Red {
    double v[kGWarps];
    long long i[kGWarps];
    double s[kGWarps][4];
};

// Block-level argmax of (v, i); thread 0 returns the result.
__device__ void block_pick(Red &r, double &v, long long &i)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
        pick(v, i, v2, i2);
    }
    __syncthreads();
    if (lane == 0) {
        r.v[w] = v;
        r.i[w] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kGWarps; ++k)
            pick(v, i, r.v[k], r.i[k]);
    }
}

// Block sums of 4 values (deterministic order); thread 0 holds the result.
__device__ void block_sum4(Red &r, double a[4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        a[c] = warp_sum_f64(a[c]);
    __syncthreads();
    if (lane == 0)
        for (int c = 0; c < 4; ++c)
            r.s[w][c] = a[c];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) {
            double t = 0.0;
            for (int k = 0; k < kGWarps; ++k)
                t += r.s[k][c];
            a[c] = t;
        }
}

// Grid-wide (value, index) argmax through per-CTA partials: every CTA reads
// the G partials after the barrier and reduces them in the same order.
__device__ void grid_pick_reduce(const double *pv, const long long *pi, int G, double &v,
                                 long long &i)
{
    __shared__ double s_v;
    __shared__ long long s_i;
    if (threadIdx.x < 32) {
        double bv = -1.0;
        long long bi = -1;
        for (int b = threadIdx.x; b < G; b += 32)
            pick(bv, bi, ldcg(pv + b), ldcg(pi + b));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            pick(bv, bi, v2, i2);
        }
        if (threadIdx.x == 0) {
            s_v = bv;
            s_i = bi;
        }
    }
    __syncthreads();
    v = s_v;
    i = s_i;
    __syncthreads();
}

// The better of two argmax candidates: the larger exact value (errors are
// non-negative doubles, compared as bit patterns), the lower node index
// among equal values (Alg. 1).  A candidate is a key, which carries the node
// (key_node) and is 0 for "none", and its exact value.
__device__ __forceinline__ bool lead_better(unsigned long long k2, double e2,
                                            unsigned long long k, double e)
{
    if (k2 == 0)
        return false;
    if (k == 0)
        return true;
    const unsigned long long b2 = dbits(e2), b = dbits(e);
    return b2 > b || (b2 == b && key_node(k2) < key_node(k));
}

// Grid-wide reductions of the per-CTA partials (4 values per CTA).  Warp 0
// loads them in parallel (lane i takes CTAs i, i + 32, ...) and combines them
// with a fixed shuffle tree, so every CTA computes the same bits.
__device__ void grid_sum4(const double *p, int G, double out[4])
{
    __shared__ double s_o[4];
    if (threadIdx.x < 32) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < G; b += 32) {
            const double2 v0 = __ldcg((const double2 *)(p + 4 * b));
            const double2 v1 = __ldcg((const double2 *)(p + 4 * b + 2));
            t[0] += v0.x;
            t[1] += v0.y;
            t[2] += v1.x;
            t[3] += v1.y;
        }
        for (int c = 0; c < 4; ++c)
            t[c] = warp_sum_f64(t[c]);
        if (threadIdx.x == 0)
            for (int c = 0; c < 4; ++c)
                s_o[c] = t[c];
    }
    __syncthreads();
    for (int c = 0; c < 4; ++c)
        out[c] = s_o[c];
    __syncthreads();
}

__device__ void grid_max4(const double *p, int G, double out[4])
{
    __shared__ double s_o[4];
    if (threadIdx.x < 32) {
        double t[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int b = threadIdx.x; b < G; b += 32) {
            const double2 v0 = __ldcg((const double2 *)(p + 4 * b));
            const double2 v1 = __ldcg((const double2 *)(p + 4 * b + 2));
            t[0] = fmax(t[0], v0.x);
            t[1] = fmax(t[1], v0.y);
            t[2] = fmax(t[2], v1.x);
            t[3] = fmax(t[3], v1.y);
        }
        for (int c = 0; c < 4; ++c)
            for (int o = 16; o > 0; o >>= 1)
                t[c] = fmax(t[c], __shfl_xor_sync(0xffffffffu, t[c], o));
        if (threadIdx.x == 0)
            for (int c = 0; c < 4; ++c)
                s_o[c] = t[c];
    }
    __syncthreads();
    for (int c = 0; c < 4; ++c)
        out[c] = s_o[c];
    __syncthreads();
}

// Squared distance with the oracle's operation order and no contraction,
// for the seed-node decisions (exact ties must resolve identically).
__device__ __forceinline__ double dist2_exact(const double *a, const double *b)
{
    const double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------
// Team layout: `ts` consecutive lanes (power of two <= 32) share one query and
// split the centres between them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int team_size(int64_t nq, int G)
{
    const int64_t lanes = (int64_t)G * kGThreads;
    int ts = 1;
    while (ts < 32 && (int64_t)(ts * 2) * nq <= lanes)
        ts *= 2;
    return ts;
}

template <typename T>
__device__ __forceinline__ T team_sum(T v, int ts)
{
    for (int o = 1; o < ts; o <<= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 error of the node at position q with the current support (nc centres).
// F(r_q) partial sums of one team lane over centres j = sub, sub + ts, ...
// (FP64), two centres per step with their loads issued together.
__device__ __forceinline__ void team_f_f64(const GreedyArgs &a, const D4 &x, int nc, int sub,
                                           int ts, double &fx, double &fy, double &fz)
{
    fx = 0.0;
    fy = 0.0;
    fz = 0.0;
    int j = sub;
    for (; j + ts < nc; j += 2 * ts) {
        const D4 c0 = ldcg(a.c64 + j), c1 = ldcg(a.c64 + j + ts);
        const D4 w0 = ldcg(a.w64 + j), w1 = ldcg(a.w64 + j + ts);
        double dx = x.x - c0.x, dy = x.y - c0.y, dz = x.z - c0.z;
        const double p0 = phi_f64_s(fma(dz, dz, fma(dy, dy, dx * dx)));
        dx = x.x - c1.x;
        dy = x.y - c1.y;
        dz = x.z - c1.z;
        const double p1 = phi_f64_s(fma(dz, dz, fma(dy, dy, dx * dx)));
        fx = fma(w1.x, p1, fma(w0.x, p0, fx));
        fy = fma(w1.y, p1, fma(w0.y, p0, fy));
        fz = fma(w1.z, p1, fma(w0.z, p0, fz));
    }
    if (j < nc) {
        const D4 c = ldcg(a.c64 + j);
        const D4 w = ldcg(a.w64 + j);
        const double dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
        const double ph = phi_f64_s(fma(dz, dz, fma(dy, dy, dx * dx)));
        fx = fma(w.x, ph, fx);
        fy = fma(w.y, ph, fy);
        fz = fma(w.z, ph, fz);
    }
    fx = team_sum(fx, ts);
    fy = team_sum(fy, ts);
    fz = team_sum(fz, ts);
}

// FP64 error of the node at position q with the current support (nc centres).
__device__ __forceinline__ double team_error_f64(const GreedyArgs &a, int q, int nc, int sub,
                                                 int ts)
{
    const D4 x = ldcg(a.xg64 + q);
    double fx, fy, fz;
    team_f_f64(a, x, nc, sub, ts, fx, fy, fz);
    const D4 d = ldcg(a.dg64 + q);
    const double ex = d.x - fx, ey = d.y - fy, ez = d.z - fz;
    return sqrt(fma(ez, ez, fma(ey, ey, ex * ex)));
}

// FP64 residual dr_q - F(r_q) of the node at position q (all lanes of the
// team return the same value).
__device__ __forceinline__ D4 team_resid_f64(const GreedyArgs &a, int q, int nc, int sub, int ts)
{
    const D4 x = ldcg(a.xg64 + q);
    double fx, fy, fz;
    team_f_f64(a, x, nc, sub, ts, fx, fy, fz);
    const D4 d = ldcg(a.dg64 + q);
    return mk4(d.x - fx, d.y - fy, d.z - fz, 0.0);
}

// Dot product of row `row` (length n, L2-coherent loads) with vector v,
// spread over the 32 lanes of a warp with four independent accumulators.
// kVShared: v lies in this CTA's shared memory (plain loads).
template <bool kVShared = false>
__device__ __forceinline__ double warp_dot(const double *row, const double *v, int p0, int n)
{
    const int lane = threadIdx.x & 31;
    auto ldv = [&](int k) { return kVShared ? v[k] : ldcg(v + k); };
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int p = p0 + lane;
    for (; p + 96 < n; p += 128) {
        const double z0 = ldcg(row + p), z1 = ldcg(row + p + 32), z2 = ldcg(row + p + 64),
                     z3 = ldcg(row + p + 96);
        const double b0 = ldv(p), b1 = ldv(p + 32), b2 = ldv(p + 64), b3 = ldv(p + 96);
        s0 = fma(z0, b0, s0);
        s1 = fma(z1, b1, s1);
        s2 = fma(z2, b2, s2);
        s3 = fma(z3, b3, s3);
    }
    for (; p < n; p += 32)
        s0 = fma(ldcg(row + p), ldv(p), s0);
    return warp_sum_f64((s0 + s1) + (s2 + s3));
}

// Same with a 3-column vector of D4 (x, y, z).
__device__ __forceinline__ void warp_dot3(const double *row, const D4 *v, int p0, int n,
                                          double &sx, double &sy, double &sz)
{
    const int lane = threadIdx.x & 31;
    double ax = 0.0, ay = 0.0, az = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
    int p = p0 + lane;
    for (; p + 32 < n; p += 64) {
        const double z0 = ldcg(row + p), z1 = ldcg(row + p + 32);
        const D4 r0 = ldcg(v + p), r1 = ldcg(v + p + 32);
        ax = fma(z0, r0.x, ax);
        ay = fma(z0, r0.y, ay);
        az = fma(z0, r0.z, az);
        bx = fma(z1, r1.x, bx);
        by = fma(z1, r1.y, by);
        bz = fma(z1, r1.z, bz);
    }
    if (p < n) {
        const double z0 = ldcg(row + p);
        const D4 r0 = ldcg(v + p);
        ax = fma(z0, r0.x, ax);
        ay = fma(z0, r0.y, ay);
        az = fma(z0, r0.z, az);
    }
    sx = warp_sum_f64(ax + bx);
    sy = warp_sum_f64(ay + by);
    sz = warp_sum_f64(az + bz);
}

struct EvalOut {
    unsigned long long key;   // argmax key over the range minus S (0 = none)
    double gmax;              // certified maximum of E over the range minus S (FP64
                              // mode, or after an FP64 re-score), else an upper bound
    double gsq;               // sum of squares of E over the range minus S
    double e_lead, b_lead;    // the leader's error and bound
    int p_lead;               // the leader's position
    long long first;          // look-ahead result (kNoRank: none)
};


// ---------------------------------------------------------------------------
// Recurrence-Cholesky append of the node at position pn (Sec. 1, RC scheme):
// with Z = L^-1 of the current nc x nc factor, b_j = phi(|r_n - r_j| / R),
//   l = Z b,  d^2 = phi(0) - l.l,  y_new = (dr_n - l.y) / d,
//   Z gains the row [-(Z^T l)^T / d, 1 / d],
//   W_j += -(Z^T l)_j / d * y_new (j < nc),  w_new = y_new / d.
// All CTAs call it; two grid barriers with s_b (double-float mode), three
// without.  Returns kAppendOk, kAppendNotSpd
// (d^2 <= kPivotMin, status latched) or kAppendTimeout.
// ---------------------------------------------------------------------------
constexpr int kAppendOk = 0, kAppendTimeout = 1, kAppendNotSpd = 2;

// 1/sqrt(x) for x > 0 in FP64 from the FP32 estimate and two Newton steps
// y <- y (3 - x y^2) / 2 (the error squares at each step: 2^-23 -> 2^-46 ->
// below FP64 rounding); about 10 FP64 instructions instead of a full FP64
// square root and division.
__device__ __forceinline__ double rsqrt_f64_newton(double x)
{
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x, y * y, 1.5);
    y = y * fma(-0.5 * x, y * y, 1.5);
    return y;
}

// Weight j of the support set into the evaluation table of the active
// precision: FP32 (centre, weight) pairs or double-float (c hi, c lo, w hi,
// w lo); .w of the weight entry is |w|_1 (FP32), used by the error bounds.
__device__ __forceinline__ void put_weight(const GreedyArgs &a, int j, const D4 &w)
{
    if (a.prec == RBF_PREC_F32X2) {
        float hx, lx, hy, ly, hz, lz;
        split_f64(w.x, hx, lx);
        split_f64(w.y, hy, ly);
        split_f64(w.z, hz, lz);
        a.cwff[2 * (size_t)a.ld + j] = make_float4(hx, hy, hz, fabsf(hx) + fabsf(hy) + fabsf(hz));
        a.cwff[3 * (size_t)a.ld + j] = make_float4(lx, ly, lz, 0.0f);
    } else if (a.prec == RBF_PREC_F32) {
        const float fx = (float)w.x, fy = (float)w.y, fz = (float)w.z;
        a.cw32[(size_t)a.ld + j] = make_float4(fx, fy, fz, fabsf(fx) + fabsf(fy) + fabsf(fz));
    }
}

// Grid unit of the grid split (split_grid) of this launch's boundary, set by
// every CTA in the prologue (double-float mode).
__shared__ double s_gunit;

// put_weight with the three components held by lanes 0-2 of the warp (all
// lanes call it): each lane splits its own component, lane 0 writes.
__device__ __forceinline__ void put_weight_lanes(const GreedyArgs &a, int j, double wc, int lane)
{
    if (a.prec == RBF_PREC_F32X2) {
        float h = 0.0f, l = 0.0f;
        if (lane < 3)
            split_f64(wc, h, l);
        const float h1 = __shfl_sync(0xffffffffu, h, 1), h2 = __shfl_sync(0xffffffffu, h, 2);
        const float l1 = __shfl_sync(0xffffffffu, l, 1), l2 = __shfl_sync(0xffffffffu, l, 2);
        if (lane == 0) {
            a.cwff[2 * (size_t)a.ld + j] = make_float4(h, h1, h2, fabsf(h) + fabsf(h1) + fabsf(h2));
            a.cwff[3 * (size_t)a.ld + j] = make_float4(l, l1, l2, 0.0f);
        }
    } else if (a.prec == RBF_PREC_F32) {
        const float f = lane < 3 ? (float)wc : 0.0f;
        const float f1 = __shfl_sync(0xffffffffu, f, 1), f2 = __shfl_sync(0xffffffffu, f, 2);
        if (lane == 0)
            a.cw32[(size_t)a.ld + j] = make_float4(f, f1, f2, fabsf(f) + fabsf(f1) + fabsf(f2));
    }
}

__device__ __forceinline__ void put_centre(const GreedyArgs &a, int j, const D4 &c)
{
    if (a.prec == RBF_PREC_F32X2) {
        float h0, l0, h1, l1, h2, l2;
        split_grid(c.x, s_gunit, h0, l0);
        split_grid(c.y, s_gunit, h1, l1);
        split_grid(c.z, s_gunit, h2, l2);
        a.cwff[j] = make_float4(h0, h1, h2, 0.0f);
        a.cwff[(size_t)a.ld + j] = make_float4(l0, l1, l2, 0.0f);
    } else if (a.prec == RBF_PREC_F32) {
        a.cw32[j] = make_float4((float)c.x, (float)c.y, (float)c.z, 0.0f);
    }
}

__device__ int chol_append(const GreedyArgs &a, Red &red, int &nc, int &use, double &min_piv,
                           int pn, int node, long long kiter, unsigned int &epoch,
                           double *s_b = nullptr)
{
    GreedyCtl *ctl = a.ctl;
    const int G = g_vg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gwarp = g_vb * kGWarps + warp, gwarps = G * kGWarps;
    // FP64 instructions cost a warp ~30 FP32 ones on this GPU, so scalar
    // FP64 work runs once per CTA (warp 0) and sums are split across warps.
    __shared__ double s_sc[8];
    // A1: b_j = phi(|r_n - r_j| / R).
    //  - s_b given (double-float evaluation; s_b is scratch shared memory of
    //    at least nc doubles): every CTA computes, in double-float on the FP32
    //    pipe, the entries its own rows of Z need (j <= its last row), so
    //    no grid barrier separates A1 from A2.  The entries carry the
    //    double-float phi's accuracy (about 2^-44 relative), the order of the
    //    FP64 factorisation's own backward error at a few hundred centres.
    //  - otherwise: FP64, centre j on CTA j mod G (FP64 work spread over every
    //    SM), then a grid barrier.
    if (s_b) {
        const int base = g_vb * kGWarps;
        int need = 0;
        if (nc > base) {
            const int last = base + ((nc - 1 - base) / gwarps) * gwarps + kGWarps - 1;
            need = min(nc, last + 1);
        }
        const float4 xh = ldcg(a.xg32 + pn), xl = ldcg(a.xgl + pn);
        for (int j = tid; j < need; j += kGThreads) {
            const float4 ch = ldcg(a.cwff + j), cl = ldcg(a.cwff + (size_t)a.ld + j);
            const ff ph = phi_ff_s(dist2_gs(xh.x, xl.x, xh.y, xl.y, xh.z, xl.z, ch.x, cl.x,
                                            ch.y, cl.y, ch.z, cl.z));
            s_b[j] = (double)ph.h + (double)ph.l;
        }
        // the table's next staging overwrites s_b with bulk (async-proxy)
        // copies: order these generic writes before them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    } else {
        const D4 xn = ldcg(a.xg64 + pn);
        for (int j = g_vb + G * tid; j < nc; j += G * kGThreads) {
            const D4 c = ldcg(a.c64 + j);
            const double dx = xn.x - c.x, dy = xn.y - c.y, dz = xn.z - c.z;
            a.bvec[j] = phi_f64_s(fma(dz, dz, fma(dy, dy, dx * dx)));
        }
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb)) return kAppendTimeout;
    }
    // A2: l = Z b (warp per row) and the partial sums of l.l and l.y (lane 0
    // of each warp accumulates its rows)
    // lane c < 4 of a warp accumulates component c of (l.l, l.y): one FP64
    // instruction per row instead of four in series
    double acc = 0.0;
    for (int i = gwarp; i < nc; i += gwarps) {
        double yc = 0.0;
        if (lane >= 1 && lane < 4)
            yc = ldcg(&a.y64[i].x + (lane - 1));
        const double s = s_b ? warp_dot<true>(a.z + (size_t)i * a.ld, s_b, 0, i + 1)
                             : warp_dot(a.z + (size_t)i * a.ld, a.bvec, 0, i + 1);
        if (lane == 0)
            a.lvec[i] = s;
        if (lane < 4)
            acc = fma(s, lane == 0 ? s : yc, acc);
    }
    if (lane < 4)
        red.s[warp][lane] = acc;
    __syncthreads();
    // the 8 warps x 4 components summed by warp 0 in a three-level tree
    if (warp == 0) {
        double t = red.s[lane >> 2][lane & 3];
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 8);
        t += __shfl_xor_sync(0xffffffffu, t, 16);
        if (lane < 4)
            (a.part + (size_t)(use & 1) * kMaxGrid * 4)[4 * g_vb + lane] = t;
    }
    if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb)) return kAppendTimeout;
    {
        // grid sums: warp c adds component c of the G partials (fixed order,
        // the same bits in every CTA)
        const double *pp = a.part + (size_t)(use & 1) * kMaxGrid * 4;
        if (warp < 4) {
            double t = 0.0;
            for (int b = lane; b < G; b += 32)
                t += ldcg(pp + 4 * b + warp);
            t = warp_sum_f64(t);
            if (lane == 0)
                s_sc[warp] = t;
        }
        __syncthreads();
        if (tid == 0) {
            const double d2 = 1.0 - s_sc[0];   // phi(0) = 1
            s_sc[4] = d2;
            if (d2 > kPivotMin) {
                const double inv_d = rsqrt_f64_newton(d2);
                const D4 dn = ldcg(a.dg64 + pn);
                s_sc[5] = inv_d;
                s_sc[0] = (dn.x - s_sc[1]) * inv_d;   // y_new = (dr_n - l.y) / d
                s_sc[1] = (dn.y - s_sc[2]) * inv_d;
                s_sc[2] = (dn.z - s_sc[3]) * inv_d;
                min_piv = fmin(min_piv, d2);
            }
        }
        __syncthreads();
    }
    ++use;
    const double d2 = s_sc[4];
    if (!(d2 > kPivotMin)) {
        if (g_vb == 0 && tid == 0)
            ctl->status = RBF_E_NOT_SPD;
        return kAppendNotSpd;
    }
    const double inv_d = s_sc[5];
    const double yx = s_sc[0], yy = s_sc[1], yz = s_sc[2];
    // A3: u = Z^T l (warp per row of Z^T); new row of Z; weight update.  The
    // new node's own entries are written by the last warp of the grid, which
    // has the fewest rows.
    // lanes 0-2 update one component of W_j each (its load issued before
    // the row product) and lane 0 assembles the table entry
    for (int j = gwarp; j < nc; j += gwarps) {
        double wc = 0.0;
        if (lane < 3)
            wc = ldcg(&a.w64[j].x + lane);
        const double s = warp_dot(a.zt + (size_t)j * a.ld, a.lvec, j, nc);
        const double zz = -s * inv_d;
        if (lane == 0) {
            a.z[(size_t)nc * a.ld + j] = zz;
            a.zt[(size_t)j * a.ld + nc] = zz;
        }
        if (lane < 3) {
            wc = fma(zz, lane == 0 ? yx : (lane == 1 ? yy : yz), wc);
            (&a.w64[j].x)[lane] = wc;
        }
        put_weight_lanes(a, j, wc, lane);
    }
    if (gwarp == gwarps - 1 && lane == 0) {
        a.z[(size_t)nc * a.ld + nc] = inv_d;
        a.zt[(size_t)nc * a.ld + nc] = inv_d;
        a.y64[nc] = mk4(yx, yy, yz, 0.0);
        const D4 wn = mk4(yx * inv_d, yy * inv_d, yz * inv_d, 0.0);   // w_new = y_new / d
        a.w64[nc] = wn;
        const D4 xc = ldcg(a.xg64 + pn);
        a.c64[nc] = xc;
        put_centre(a, nc, xc);
        put_weight(a, nc, wn);
        a.spos[nc] = pn;
        a.in_s[pn] = 1;
        a.sel_idx[nc] = node;
        if (a.sel_iter)
            a.sel_iter[nc] = kiter;
    }
    if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb)) return kAppendTimeout;
    ++nc;
    return kAppendOk;
}


// ---------------------------------------------------------------------------
// Block append of K >= 2 nodes (positions pk_pos[0..K), in that order): the
// same factor as K single appends, in three grid barriers.  With Z = L^-1 of
// the current n x n factor and y = Z dX_S:
//   B = Phi(S, new) (n x K),  Lambda = Z B,  M = Phi(new, new) - Lambda^T Lambda,
//   L22 = chol(M),  Z22 = L22^-1,  y_new = Z22 (dX_new - Lambda^T y),
//   w_new = Z22^T y_new,  U = Z^T Lambda,
//   Z gains the rows [-Z22 U^T, Z22],  W_S -= U w_new.
// The pivots of M are the d^2 of the single appends; at the first one <=
// kPivotMin the nodes before it are appended and kAppendNotSpd is returned.
// Lanes of a warp split as (jl, kl) = (lane / K', lane % K'): a warp's row
// product reads each Z entry once for all K columns.  The K x K work (one
// warp) and the grid sums are done by every CTA in the same order, so every
// CTA holds the same bits.  `nc` grows by the number appended.
// ---------------------------------------------------------------------------
__device__ int chol_append_block(const GreedyArgs &a, int &nc, double &min_piv, int K,
                                 const int *pk_pos, const int *pk_node, long long kiter,
                                 unsigned int &epoch)
{
    GreedyCtl *ctl = a.ctl;
    const int G = g_vg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtid = g_vb * kGThreads + tid, gthreads = G * kGThreads;
    const int gwarp = g_vb * kGWarps + warp, gwarps = G * kGWarps;
    const int n = nc;
    const int KP = K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : 16;   // K' (power of two)
    const int lgKP = K <= 2 ? 1 : K <= 4 ? 2 : K <= 8 ? 3 : 4;
    const int J = 32 / KP;
    const int kl = lane & (KP - 1), jl = lane >> lgKP;
    const int V = KP * KP + 3 * KP;
    __shared__ double s_acc[kBlkV];
    __shared__ double s_l[kMaxPeaks][kMaxPeaks + 1];   // M, overwritten by L22 below the diagonal
    __shared__ double s_z[kMaxPeaks][kMaxPeaks + 1];   // Z22
    __shared__ double s_inv[kMaxPeaks];
    __shared__ double s_y[kMaxPeaks][3], s_w[kMaxPeaks][3];
    __shared__ int s_keff;

    // B1: B[j][k] = phi(|r_new_k - r_j| / R) (zero for k >= K) and Phi(new, new)
    for (int t = gtid; t < n * KP; t += gthreads) {
        const int j = t >> lgKP, k = t & (KP - 1);
        double b = 0.0;
        if (k < K) {
            const D4 x = ldcg(a.xg64 + pk_pos[k]), c = ldcg(a.c64 + j);
            const double dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
            b = phi_f64_s(fma(dz, dz, fma(dy, dy, dx * dx)));
        }
        a.bmat[t] = b;
    }
    if (gtid < K * K) {
        const int k = gtid / K, l = gtid - k * K;
        const D4 x = ldcg(a.xg64 + pk_pos[k]), c = ldcg(a.xg64 + pk_pos[l]);
        const double dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
        a.cmat[gtid] = phi_f64_s(fma(dz, dz, fma(dy, dy, dx * dx)));
    }
    if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
        return kAppendTimeout;

    // B2: Lambda = Z B (warp per row), with the partial sums of Lambda^T
    // Lambda (entry (kl, l), l = jl + t J) and of Lambda^T y (entry (kl, c),
    // c = jl + t J < 3) kept by the lane that owns them
    double gacc[kMaxPeaks / 2], yacc[2];
#pragma unroll
    for (int t = 0; t < kMaxPeaks / 2; ++t)
        gacc[t] = 0.0;
    yacc[0] = yacc[1] = 0.0;
    for (int i = gwarp; i < n; i += gwarps) {
        const double *zr = a.z + (size_t)i * a.ld;
        double s = 0.0;
        for (int j = jl; j <= i; j += J)
            s = fma(ldcg(zr + j), ldcg(a.bmat + (size_t)j * KP + kl), s);
        for (int o = KP; o < 32; o <<= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (jl == 0)
            a.lmat[(size_t)i * KP + kl] = s;
        const D4 y = ldcg(a.y64 + i);
#pragma unroll
        for (int t = 0; t < kMaxPeaks / 2; ++t) {
            if (t * J >= KP)
                break;
            const int l = jl + t * J;
            const double sl = __shfl_sync(0xffffffffu, s, l < KP ? l : 0);
            if (l < KP)
                gacc[t] = fma(s, sl, gacc[t]);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = jl + t * J;
            if (c < 3)
                yacc[t] = fma(s, c == 0 ? y.x : c == 1 ? y.y : y.z, yacc[t]);
        }
    }
    for (int v = tid; v < V; v += kGThreads)
        s_acc[v] = 0.0;
    __syncthreads();
    for (int w = 0; w < kGWarps; ++w) {   // warps in order: the same sums in every run
        if (warp == w) {
#pragma unroll
            for (int t = 0; t < kMaxPeaks / 2; ++t) {
                const int l = jl + t * J;
                if (t * J < KP && l < KP)
                    s_acc[kl * KP + l] += gacc[t];
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int c = jl + t * J;
                if (c < 3)
                    s_acc[KP * KP + 3 * kl + c] += yacc[t];
            }
        }
        __syncthreads();
    }
    for (int v = tid; v < V; v += kGThreads)
        a.bpart[(size_t)g_vb * kBlkV + v] = s_acc[v];
    if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
        return kAppendTimeout;
    // grid sums: the CTAs split into nseg fixed segments; thread (seg, v)
    // adds its segment's partials of value v (independent loads), then each
    // value's segment sums are added in segment order (the same bits in every
    // CTA)
    {
        __shared__ double s_seg[kBlkV];   // nseg * V <= kBlkV for every K'
        const int nseg = min(kBlkSeg, max(1, kGThreads / V));
        const int per = (G + nseg - 1) / nseg;
        for (int t = tid; t < nseg * V; t += kGThreads) {
            const int seg = t / V, v = t - seg * V;
            const int b0 = seg * per, b1 = min(G, b0 + per);
            double s0 = 0.0, s1 = 0.0;
            int b = b0;
#pragma unroll 4
            for (; b + 1 < b1; b += 2) {
                s0 += ldcg(a.bpart + (size_t)b * kBlkV + v);
                s1 += ldcg(a.bpart + (size_t)(b + 1) * kBlkV + v);
            }
            if (b < b1)
                s0 += ldcg(a.bpart + (size_t)b * kBlkV + v);
            s_seg[t] = s0 + s1;
        }
        __syncthreads();
        for (int v = tid; v < V; v += kGThreads) {
            double t = 0.0;
            for (int seg = 0; seg < nseg; ++seg)
                t += s_seg[seg * V + v];
            s_acc[v] = t;
        }
        __syncthreads();
    }

    // B3 (warp 0): L22 = chol(M) row by row, Z22, y_new, w_new
    if (warp == 0) {
        for (int t = lane; t < K * K; t += 32) {
            const int k = t / K, l = t - k * K;
            if (l <= k)
                s_l[k][l] = ldcg(a.cmat + t) - s_acc[k * KP + l];
        }
        if (lane < K) {   // dX_new - Lambda^T y, row `lane`
            const D4 dn = ldcg(a.dg64 + pk_pos[lane]);
            const double *ly = s_acc + KP * KP + 3 * lane;
            s_y[lane][0] = dn.x - ly[0];
            s_y[lane][1] = dn.y - ly[1];
            s_y[lane][2] = dn.z - ly[2];
        }
        __syncwarp();
        int keff = K;
        for (int k = 0; k < K; ++k) {
            const double d2 = s_l[k][k];
            if (!(d2 > kPivotMin)) {
                keff = k;
                break;
            }
            if (lane == 0) {
                s_inv[k] = rsqrt_f64_newton(d2);
                min_piv = fmin(min_piv, d2);
            }
            __syncwarp();
            const double inv = s_inv[k];
            if (lane > k && lane < K)
                s_l[lane][k] *= inv;
            __syncwarp();
            if (lane > k && lane < K) {
                const double lk = s_l[lane][k];
                for (int j = k + 1; j <= lane; ++j)
                    s_l[lane][j] = fma(-lk, s_l[j][k], s_l[lane][j]);
            }
            __syncwarp();
        }
        if (lane < keff) {   // column `lane` of Z22 by forward substitution
            const int j = lane;
            s_z[j][j] = s_inv[j];
            for (int i = j + 1; i < keff; ++i) {
                double t = 0.0;
                for (int m = j; m < i; ++m)
                    t = fma(s_l[i][m], s_z[m][j], t);
                s_z[i][j] = -t * s_inv[i];
            }
        }
        __syncwarp();
        double r0 = 0.0, r1 = 0.0, r2 = 0.0;
        if (lane < keff) {   // y_new = Z22 (dX_new - Lambda^T y), row `lane`
            const int i = lane;
            for (int m = 0; m <= i; ++m) {
                r0 = fma(s_z[i][m], s_y[m][0], r0);
                r1 = fma(s_z[i][m], s_y[m][1], r1);
                r2 = fma(s_z[i][m], s_y[m][2], r2);
            }
        }
        __syncwarp();
        if (lane < keff) {
            s_y[lane][0] = r0;
            s_y[lane][1] = r1;
            s_y[lane][2] = r2;
        }
        __syncwarp();
        if (lane < keff) {   // w_new = Z22^T y_new, row `lane`
            const int k = lane;
            double w0 = 0.0, w1 = 0.0, w2 = 0.0;
            for (int i = k; i < keff; ++i) {
                w0 = fma(s_z[i][k], s_y[i][0], w0);
                w1 = fma(s_z[i][k], s_y[i][1], w1);
                w2 = fma(s_z[i][k], s_y[i][2], w2);
            }
            s_w[k][0] = w0;
            s_w[k][1] = w1;
            s_w[k][2] = w2;
        }
        if (lane == 0)
            s_keff = keff;
    }
    __syncthreads();
    const int keff = s_keff;
    if (keff == 0) {
        if (g_vb == 0 && tid == 0)
            ctl->status = RBF_E_NOT_SPD;
        return kAppendNotSpd;
    }

    // B4: U = Z^T Lambda (warp per row j of Z^T), the new rows' entries
    // -Z22 U^T in column j, and W_j -= U_j w_new
    for (int j = gwarp; j < n; j += gwarps) {
        const double *ztr = a.zt + (size_t)j * a.ld;
        double s = 0.0;
        for (int i = j + jl; i < n; i += J)
            s = fma(ldcg(ztr + i), ldcg(a.lmat + (size_t)i * KP + kl), s);
        for (int o = KP; o < 32; o <<= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        double z21 = 0.0;
        for (int l = 0; l < KP; ++l) {
            const double ul = __shfl_sync(0xffffffffu, s, l);
            if (l <= kl && kl < keff)
                z21 = fma(s_z[kl][l], ul, z21);
        }
        double px = 0.0, py = 0.0, pz = 0.0;
        if (kl < keff) {
            px = s * s_w[kl][0];
            py = s * s_w[kl][1];
            pz = s * s_w[kl][2];
        }
        for (int o = 1; o < KP; o <<= 1) {
            px += __shfl_xor_sync(0xffffffffu, px, o);
            py += __shfl_xor_sync(0xffffffffu, py, o);
            pz += __shfl_xor_sync(0xffffffffu, pz, o);
        }
        if (jl == 0 && kl < keff) {
            a.z[(size_t)(n + kl) * a.ld + j] = -z21;
            a.zt[(size_t)j * a.ld + n + kl] = -z21;
        }
        if (lane == 0) {
            D4 w = ldcg(a.w64 + j);
            w.x -= px;
            w.y -= py;
            w.z -= pz;
            a.w64[j] = w;
            put_weight(a, j, w);
        }
    }
    // the new nodes' own entries: the last warp of the grid, lane k for node k
    if (gwarp == gwarps - 1 && lane < keff) {
        const int k = lane;
        for (int l = 0; l <= k; ++l) {
            a.z[(size_t)(n + k) * a.ld + n + l] = s_z[k][l];
            a.zt[(size_t)(n + l) * a.ld + n + k] = s_z[k][l];
        }
        a.y64[n + k] = mk4(s_y[k][0], s_y[k][1], s_y[k][2], 0.0);
        const D4 wn = mk4(s_w[k][0], s_w[k][1], s_w[k][2], 0.0);
        a.w64[n + k] = wn;
        const int pn = pk_pos[k];
        const D4 xc = ldcg(a.xg64 + pn);
        a.c64[n + k] = xc;
        put_centre(a, n + k, xc);
        put_weight(a, n + k, wn);
        a.spos[n + k] = pn;
        a.in_s[pn] = 1;
        a.sel_idx[n + k] = pk_node[k];
        if (a.sel_iter)
            a.sel_iter[n + k] = kiter;
    }
    if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
        return kAppendTimeout;
    nc = n + keff;
    if (keff < K) {
        if (g_vb == 0 && tid == 0)
            ctl->status = RBF_E_NOT_SPD;
        return kAppendNotSpd;
    }
    return kAppendOk;
}

// ---------------------------------------------------------------------------
// FP64 iterative refinement of the support weights (Sec. 2: Phi_SS is SPD,
// solved through its Cholesky factor): `steps` times
//   r = dX_S - Phi_SS W (recomputed from coordinates),  W += Z^T (Z r),
// then the residual of the final W; `maxres` = max_j |r_j|_inf.  Support node
// j sits at position spos[j] (identity when spos is null).  All CTAs call it.
// ---------------------------------------------------------------------------
__device__ bool refine_weights(const GreedyArgs &a, Red &red, int nc, int &use,
                               unsigned int &epoch, int steps, const int32_t *spos, D4 *rvec,
                               D4 *tvec, double &maxres)
{
    GreedyCtl *ctl = a.ctl;
    const int G = g_vg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtid = g_vb * kGThreads + tid;
    const int gthreads = G * kGThreads;
    const int gwarp = g_vb * kGWarps + warp, gwarps = G * kGWarps;
    const int ts = team_size(nc, G);
    const int sub = lane & (ts - 1);
    const int team = gtid / ts, nteams = gthreads / ts;
    const int rounds = (nc + nteams - 1) / nteams;
    for (int step = 0; step <= steps; ++step) {
        double lmax = 0.0;
        for (int it = 0; it < rounds; ++it) {
            const int q = team + it * nteams;
            const bool act = q < nc;
            const int pos = act ? (spos ? ldcg(spos + q) : q) : (spos ? ldcg(spos) : 0);
            const D4 r = team_resid_f64(a, pos, nc, sub, ts);
            if (act && sub == 0) {
                rvec[q] = r;
                lmax = fmax(lmax, fmax(fabs(r.x), fmax(fabs(r.y), fabs(r.z))));
            }
        }
        for (int o = 16; o > 0; o >>= 1)
            lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        __syncthreads();
        if (lane == 0)
            red.v[warp] = lmax;
        __syncthreads();
        double *pp = a.part + (size_t)(use & 1) * kMaxGrid * 4;
        if (tid == 0) {
            for (int k = 1; k < kGWarps; ++k)
                lmax = fmax(lmax, red.v[k]);
            pp[4 * g_vb] = lmax;
        }
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
            return false;
        {
            double g4[4];
            grid_max4(pp, G, g4);
            maxres = g4[0];
            ++use;
        }
        if (step == steps)
            break;
        // t = Z r (3 right-hand sides, warp per row)
        for (int i = gwarp; i < nc; i += gwarps) {
            double sx, sy, sz;
            warp_dot3(a.z + (size_t)i * a.ld, rvec, 0, i + 1, sx, sy, sz);
            if (lane == 0)
                tvec[i] = mk4(sx, sy, sz, 0.0);
        }
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
            return false;
        // W += Z^T t
        for (int j = gwarp; j < nc; j += gwarps) {
            double sx, sy, sz;
            warp_dot3(a.zt + (size_t)j * a.ld, tvec, j, nc, sx, sy, sz);
            if (lane == 0) {
                D4 w = ldcg(a.w64 + j);
                w.x += sx;
                w.y += sy;
                w.z += sz;
                a.w64[j] = w;
            }
        }
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
            return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Barrier placement.  Thread 0 of CTA 0 times kBarCalRounds grid barriers on
// each candidate flag array of the control block; the fastest is published
// through the control block's own barrier and serves the rest of the launch
// (g_bar).  Every candidate's flags start at 0 (the host clears the control
// block), so each has its own epoch; `epoch` continues from the chosen one's
// kBarCalRounds and `extra` counts the other barriers passed.  Grids outside
// [kBarCalMinCtas, kBarCandWords] keep the control block's barrier.  All
// CTAs call it before their first grid barrier; false on a barrier timeout.
// ---------------------------------------------------------------------------
__device__ bool place_barrier(const GreedyArgs &a, int G, unsigned int &epoch, long long &extra)
{
    GreedyCtl *ctl = a.ctl;
    if (G < kBarCalMinCtas || G > kBarCandWords)
        return true;
    unsigned long long best = ~0ull;
    int pick = 0;
    for (int k = 0; k < kBarCand; ++k) {
        GridBar *cb = reinterpret_cast<GridBar *>(ctl->bar_cand[k]);
        unsigned int ek = 0;
        const unsigned long long t0 = clock64();
        for (int r = 0; r < kBarCalRounds; ++r)
            if (!grid_barrier(cb, &ctl->status, (unsigned)G, a.barrier_ns, ek, (unsigned)g_vb))
                return false;
        const unsigned long long dt = clock64() - t0;
        if (dt < best) {
            best = dt;
            pick = k;
        }
    }
    if (g_vb == 0 && threadIdx.x == 0)
        ctl->bar_pick = pick;
    if (!grid_barrier(&ctl->bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb))
        return false;   // the control block's barrier publishes bar_pick
    if (threadIdx.x == 0)
        g_bar = reinterpret_cast<GridBar *>(ctl->bar_cand[ldcg(&ctl->bar_pick)]);
    __syncthreads();
    extra += (long long)epoch + (long long)(kBarCand - 1) * kBarCalRounds;
    epoch = kBarCalRounds;
    return true;
}

// ---------------------------------------------------------------------------
// The persistent greedy: one problem on the CTAs g_vb = 0 .. g_vg - 1.
// kPeaks: the peak-selection variant (a.peaks > 1) is compiled in.
// ---------------------------------------------------------------------------
template <bool kPeaks>
__device__ __forceinline__ void greedy_body(const GreedyArgs &a)
{
    extern __shared__ float4 s_cw[];
    __shared__ Red red;
    __shared__ float s_wabs;
    __shared__ __align__(8) unsigned long long s_mbar;
    unsigned mbar_phase = 0;
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar, 1);
        g_bar_wait_ns = 0;
        g_bar = &a.ctl->bar;
    }
    __syncthreads();
    GreedyCtl *ctl = a.ctl;
    const int G = g_vg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtid = g_vb * kGThreads + tid;
    const int gthreads = G * kGThreads;
    const int nb = a.nb, m = a.m;
    int use = 0;   // partial-buffer use counter (double buffering)
    unsigned int epoch = 0;   // grid barriers passed
    // phase clock of CTA 0, thread 0: 0 prologue, 1 evaluation pass 1,
    // 2 evaluation pass 2 + reductions, 3 appends, 4 refinement, 5 other
    unsigned long long ph_acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long ph_t = globaltimer_ns();
    int ph_cur = 0;
    auto phase = [&](int nx) {
        if (g_vb == 0 && threadIdx.x == 0) {
            const unsigned long long now = globaltimer_ns();
            ph_acc[ph_cur] += now - ph_t;
            ph_t = now;
            ph_cur = nx;
        }
    };
    auto part = [&](int u) { return a.part + (size_t)(u & 1) * kMaxGrid * 4; };
    auto parti = [&](int u) { return a.parti + (size_t)(u & 1) * kMaxGrid; };
#define GSYNC()                                                                   \
    do {                                                                          \
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb)) \
            return;                                                               \
    } while (0)
#define GSYNC_B()                                                                 \
    do {                                                                          \
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb)) \
            return false;                                                         \
    } while (0)

    // Failure-path test: CTA 0 leaves before the first barrier, so the other
    // CTAs' bounded waits run out and the launch returns RBF_E_TIMEOUT.
    if ((a.flags & RBF_FLAG_TEST_BARRIER_TIMEOUT) && g_vb == 0)
        return;

    // ---------------- barrier placement ------------------------------------
    long long bar_extra = 0;   // barriers passed that `epoch` does not count
    if (!place_barrier(a, G, epoch, bar_extra))
        return;

    // ---------------- prologue: group-ordered packing ----------------------
    double dmax = 0.0, xmax = 0.0;
    int bad = 0;
    for (int p = gtid; p < nb; p += gthreads) {
        const int node = a.perm[p];
        const int pos = goff(p % m, nb, m) + p / m;
        a.node_of_pos[pos] = node;
        a.pos_of_node[node] = pos;
        const double x = a.xb[3 * node] * a.inv_r, y = a.xb[3 * node + 1] * a.inv_r,
                     z = a.xb[3 * node + 2] * a.inv_r;
        const double d0 = a.db[3 * node], d1 = a.db[3 * node + 1], d2 = a.db[3 * node + 2];
        a.xg64[pos] = mk4(x, y, z, 0.0);
        {
            float h0, l0, h1, l1, h2, l2;
            if (a.prec != RBF_PREC_F32X2) {
                // FP32 copy (FP32 mode) and its remainders; double-float mode
                // writes the grid split once the maximum |x| is known
                a.xg32[pos] = make_float4((float)x, (float)y, (float)z, 0.0f);
                split_f64(x, h0, l0);
                split_f64(y, h1, l1);
                split_f64(z, h2, l2);
                a.xgl[pos] = make_float4(l0, l1, l2, 0.0f);
            }
            split_f64(d0, h0, l0);
            split_f64(d1, h1, l1);
            split_f64(d2, h2, l2);
            a.dgh[pos] = make_float4(h0, h1, h2, 0.0f);
            a.dgl[pos] = make_float4(l0, l1, l2, 0.0f);
        }
        a.dg64[pos] = mk4(d0, d1, d2, 0.0);
        a.in_s[pos] = 0;
        if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(d0) || !isfinite(d1) ||
            !isfinite(d2))
            bad = 1;
        dmax = fmax(dmax, d0 * d0 + d1 * d1 + d2 * d2);
        xmax = fmax(xmax, fmax(fabs(x), fmax(fabs(y), fabs(z))));
    }
    {
        double mx[3] = {dmax, xmax, (double)bad};
        for (int o = 16; o > 0; o >>= 1)
            for (int c = 0; c < 3; ++c)
                mx[c] = fmax(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        __syncthreads();
        if (lane == 0)
            for (int c = 0; c < 3; ++c)
                red.s[warp][c] = mx[c];
        __syncthreads();
        if (tid == 0) {
            for (int k = 1; k < kGWarps; ++k)
                for (int c = 0; c < 3; ++c)
                    mx[c] = fmax(mx[c], red.s[k][c]);
            double *pp = part(use) + 4 * g_vb;
            pp[0] = mx[0];
            pp[1] = mx[1];
            pp[2] = mx[2];
            pp[3] = 0.0;
        }
    }
    GSYNC();
    double g4[4];
    grid_max4(part(use), G, g4);
    ++use;
    if (g4[2] > 0.0) {
        if (g_vb == 0 && tid == 0)
            ctl->status = RBF_E_NONFINITE;
        return;   // every CTA sees the same flag
    }
    const double estar = a.tol_mode == 1 ? a.tol * sqrt(g4[0]) : a.tol;
    const float xscale = (float)g4[1];
    if (a.prec == RBF_PREC_F32X2) {
        // grid split of the scaled coordinates (exact differences in the
        // pair distances); visible to every CTA after the seed search's
        // grid barriers, before the first append reads it
        if (tid == 0)
            s_gunit = grid_unit(g4[1]);
        __syncthreads();
        for (int p = gtid; p < nb; p += gthreads) {
            const D4 x = ldcg(a.xg64 + p);
            float h0, l0, h1, l1, h2, l2;
            split_grid(x.x, s_gunit, h0, l0);
            split_grid(x.y, s_gunit, h1, l1);
            split_grid(x.z, s_gunit, h2, l2);
            a.xg32[p] = make_float4(h0, h1, h2, 0.0f);
            a.xgl[p] = make_float4(l0, l1, l2, 0.0f);
        }
    }

    // ---------------- seed nodes (lowest index on ties) ---------------------
    int seeds[3];
    for (int s = 0; s < 3; ++s) {
        double bv = -1.0;
        long long bi = -1;
        for (int n = gtid; n < nb; n += gthreads) {
            double v;
            if (s == 0) {
                const double *d = a.db + 3 * n;
                v = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                              __dmul_rn(d[2], d[2]));
            } else if (s == 1) {
                v = dist2_exact(a.xb + 3 * n, a.xb + 3 * seeds[0]);
            } else {
                v = fmin(dist2_exact(a.xb + 3 * n, a.xb + 3 * seeds[0]),
                         dist2_exact(a.xb + 3 * n, a.xb + 3 * seeds[1]));
            }
            pick(bv, bi, v, n);
        }
        block_pick(red, bv, bi);
        if (tid == 0) {
            part(use)[g_vb] = bv;
            parti(use)[g_vb] = bi;
        }
        GSYNC();
        double v;
        long long i;
        grid_pick_reduce(part(use), parti(use), G, v, i);
        ++use;
        seeds[s] = (int)i;
    }

    int nc = 0;
    double min_piv = INFINITY;
    int staged_nc = -1;   // nc of the centre table last staged in shared memory
    // Scratch for the append's phi row: the shared-memory centre table (64
    // bytes per centre in double-float mode, so room for 8 doubles per
    // staged centre).  An append changes nc, after which the table is staged
    // again; staged_nc is reset after every append that used the scratch, so
    // a failed one cannot leave a clobbered table marked current.
    auto bscratch = [&]() -> double * {
        return a.prec == RBF_PREC_F32X2 && nc <= 8 * a.smem_cap
                   ? reinterpret_cast<double *>(s_cw) : nullptr;
    };

    for (int s = 0; s < 3; ++s) {
        const int pn = ldcg(a.pos_of_node + seeds[s]);
        const int ar = chol_append(a, red, nc, use, min_piv, pn, seeds[s], -1, epoch, bscratch());
        staged_nc = -1;
        if (ar != kAppendOk) {
            if (g_vb == 0 && tid == 0) {
                ctl->nc = nc;
                ctl->min_pivot = min_piv;
            }
            return;
        }
    }

    phase(5);
    // ---------------- error evaluation over a position range ---------------
    int ev = 0;                      // evaluation counter
    long long pairs32 = 0, pairs64 = 0, pairsff = 0;
    unsigned long long rescored_local = 0;
    // Evaluates E at positions [p0, p1) with the current weights.  With
    // `argmax`, the largest E among nodes not in S (lowest node index on
    // ties) comes back as a key; `out.gmax` is the certified maximum of E over
    // the range (nodes of S excluded: their error is the FP64 interpolation
    // residual) and `out.gsq` the sum of squares.  `force64` evaluates every
    // pair in FP64 whatever the precision mode.
    // With look >= 0 (a look-ahead over all nodes), also the smallest cyclic
    // rank (position - look) mod N_b of a node outside S whose error may
    // exceed E* (upper bound E~ + beta > E*).
    // With `cached`, nothing is recomputed: the pass reads the errors and
    // bounds the last evaluations stored (valid while the weights are
    // unchanged, i.e. until the next append).
    auto evaluate = [&](int p0, int p1, bool argmax, bool force64, EvalOut &out, int look,
                        bool cached) -> bool {
        phase(1);
        const int nq = p1 - p0;
        const int ts = team_size(nq, G);
        const int sub = lane & (ts - 1);
        const int team = gtid / ts, nteams = gthreads / ts;
        const int rounds = (nq + nteams - 1) / nteams;
        unsigned long long key = 0;
        // maxima and bounds are non-negative doubles kept as bit patterns,
        // compared on the integer pipe (dbits)
        unsigned long long mxb = 0;          // largest E (E~ in screened modes)
        float lsq = 0.0f;                    // sum of E^2 (RMS diagnostic)
        double e_lead = 0.0, b_lead = 0.0;   // error and bound of this thread's leader
        long long p_lead = -1;                // its position
        long long first = kNoRank;            // look-ahead rank
        const bool screened = !(a.prec == RBF_PREC_F64 || force64);
        const unsigned long long estar_b = dbits(estar);
        // top two upper bounds E~ + beta of this thread's nodes (screened
        // modes; 0 = none, a real bound is > 0)
        unsigned long long u1 = 0, u2 = 0;
        long long n1 = -1;
        if (cached) {
            phase(look >= 0 ? 11 : 8);
            for (int it = 0; it < rounds; ++it) {
                const int q = p0 + team + it * nteams;
                if (q < p1 && sub == 0 && !ldcg(a.in_s + q)) {
                    const double e = ldcg(a.e64 + q);
                    const float bf = screened ? ldcg(a.u32 + q) : 0.0f;
                    const unsigned long long upb = dbits(e + (double)bf);
                    if (look >= 0 && upb > estar_b)
                        first = min(first, (long long)((q - look + nb) % nb));
                    mxb = max(mxb, dbits(e));
                    lsq = fmaf((float)e, (float)e, lsq);
                    if (upb > u1) {
                        u2 = u1;
                        u1 = upb;
                        n1 = ldcg(a.node_of_pos + q);
                    } else if (upb > u2) {
                        u2 = upb;
                    }
                }
            }
        } else if (!screened) {
            for (int it = 0; it < rounds; ++it) {
                const int q = p0 + team + it * nteams;
                const bool act = q < p1;
                const double e = team_error_f64(a, act ? q : p0, nc, sub, ts);
                if (act && sub == 0 && !ldcg(a.in_s + q)) {
                    a.e64[q] = e;
                    mxb = max(mxb, dbits(e));
                    lsq = fmaf((float)e, (float)e, lsq);
                    if (look >= 0 && e > estar)
                        first = min(first, (long long)((q - look + nb) % nb));
                    if (argmax) {
                        const unsigned long long k2 = key_f64(e, ldcg(a.node_of_pos + q));
                        if (lead_better(k2, e, key, e_lead)) {
                            key = k2;
                            e_lead = e;
                            b_lead = 0.0;
                            p_lead = q;
                        }
                    }
                }
            }
            if (g_vb == 0 && tid == 0)
                pairs64 += (long long)nq * nc;
        } else {
            // ---- pass 1: FP32 or double-float errors E~ with a bound beta,
            // |E~ - E| <= beta; e64[q] = E~, u32[q] = beta.  The centre table
            // is staged in shared memory by bulk (TMA) copies of its planes.
            const bool use_ff = a.prec == RBF_PREC_F32X2;
            const bool smem = nc <= a.smem_cap;
            phase(7);
            // plane stride: nc in shared memory, ld in global memory
            const int planes = use_ff ? 4 : 2, wplane = use_ff ? 2 : 1;
            const int pst = smem ? nc : a.ld;
            // the table (and |w|_1) changes only with an append, which grows
            // nc: after idle iterations the staged copy is still current
            const bool fresh = nc != staged_nc;
            if (smem && fresh) {
                const float4 *src = use_ff ? a.cwff : a.cw32;
                const unsigned pbytes = (unsigned)(sizeof(float4) * nc);
                __syncthreads();   // previous readers of the table are done
                if (tid == 0) {
                    mbar_expect(&s_mbar, pbytes * planes);
                    for (int k = 0; k < planes; ++k)
                        bulk_copy_g2s(s_cw + (size_t)k * nc, src + (size_t)k * a.ld, pbytes,
                                      &s_mbar);
                }
                const bool got = mbar_wait(&s_mbar, mbar_phase, a.barrier_ns);
                if (!got) {
                    // give the copy in flight a second bounded wait before leaving
                    atomicExch(&ctl->status, (int)RBF_E_TIMEOUT);
                    mbar_wait(&s_mbar, mbar_phase, a.barrier_ns);
                    return false;
                }
                mbar_phase ^= 1u;
            }
            if (fresh) {
                if (tid < 32) {
                    float t = 0.0f;
                    for (int j = tid; j < nc; j += 32)
                        // .w of the weight plane (plane 2 double-float, 1 FP32) = |w|_1
                        t += smem ? s_cw[(size_t)wplane * nc + j].w
                                  : ldcg((use_ff ? a.cwff : a.cw32) + (size_t)wplane * a.ld + j).w;
                    t = team_sum(t, 32);
                    if (tid == 0)
                        s_wabs = t;
                }
                staged_nc = nc;
                __syncthreads();
            }
            phase(look >= 0 ? 11 : 8);
            // terms per lane, team levels and the rounding-up factor of the
            // bounds (see the derivation at kU32)
            const int n_l = (nc + ts - 1) / ts;
            const float lg_ts = (float)(31 - __clz(ts));
            const float b_up =
                1.0f + (2.0f * (float)n_l + 2.0f * lg_ts + (float)nc * (1.0f / 32.0f) + 40.0f) * kU32;
            if (!use_ff) {
                const float4 *cw = smem ? s_cw : a.cw32;
                const float c_sb = (float)n_l + lg_ts + 10.0f;
                const float coord_term = (7.32f * xscale + 4.5f) * s_wabs;
                for (int it = 0; it < rounds; ++it) {
                    const int q = p0 + team + it * nteams;
                    const bool act = q < p1;
                    const float4 x = ldcg(a.xg32 + (act ? q : p0));
                    float fx = 0.0f, fy = 0.0f, fz = 0.0f, sb = 0.0f;
                    for (int j = sub; j < nc; j += ts) {
                        const float4 c = smem ? cw[j] : ldcg(cw + j);
                        const float4 w = smem ? cw[pst + j] : ldcg(cw + pst + j);
                        const float dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
                        const float ph = phi_f32_s(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                        fx = fmaf(w.x, ph, fx);
                        fy = fmaf(w.y, ph, fy);
                        fz = fmaf(w.z, ph, fz);
                        sb = fmaf(w.w, ph, sb);
                    }
                    fx = team_sum(fx, ts);
                    fy = team_sum(fy, ts);
                    fz = team_sum(fz, ts);
                    sb = team_sum(sb, ts);
                    if (act && sub == 0 && !ldcg(a.in_s + q)) {
                        const D4 d = ldcg(a.dg64 + q);
                        const float ex = (float)d.x - fx, ey = (float)d.y - fy,
                                    ez = (float)d.z - fz;
                        const float e = sqrtf(fmaf(ez, ez, fmaf(ey, ey, ex * ex)));
                        const float dabs = (float)(fabs(d.x) + fabs(d.y) + fabs(d.z));
                        // bound of |E32 - E|: rounding of phi and of the sums
                        // (proportional to sum |w| phi), of the coordinates
                        // (max|x|/R * sum |w|), of the displacement and of E
                        const float beta =
                            kU32 * (c_sb * sb + dabs + coord_term + 4.24f * e) * b_up + 1e-30f;
                        a.u32[q] = beta;
                        a.e64[q] = (double)e;
                        const unsigned long long upb = dbits((double)e + (double)beta);
                        if (look >= 0 && upb > estar_b)
                            first = min(first, (long long)((q - look + nb) % nb));
                        mxb = max(mxb, dbits((double)e));
                        lsq = fmaf(e, e, lsq);
                        if (argmax) {
                            const unsigned long long k2 = key_f64((double)e, ldcg(a.node_of_pos + q));
                            if (lead_better(k2, (double)e, key, e_lead)) {
                                key = k2;
                                e_lead = (double)e;
                                b_lead = (double)beta;
                                p_lead = q;
                            }
                        }
                        if (upb > u1) {
                            u2 = u1;
                            u1 = upb;
                            n1 = ldcg(a.node_of_pos + q);
                        } else if (upb > u2) {
                            u2 = upb;
                        }
                    }
                }
                if (g_vb == 0 && tid == 0)
                    pairs32 += (long long)nq * nc;
            } else {
                const float4 *cw = smem ? s_cw : a.cwff;
                // wide teams: two warps per node when the group leaves room
                // (at most one node per warp pair of the grid), which halves
                // each lane's chain of pairs -- the pass is latency-bound
                const bool wide = (int64_t)nq * 64 <= (int64_t)gthreads;
                const int tsw = wide ? 64 : ts;
                const int subw = wide ? (tid & 63) : sub;
                const int teamw = wide ? (gtid >> 6) : team;
                const int nteamsw = wide ? (gthreads >> 6) : nteams;
                const int roundsw = (nq + nteamsw - 1) / nteamsw;
                const int n_lw = (nc + tsw - 1) / tsw;
                const float lg_w = (float)(31 - __clz(tsw));
                const float b_upw =
                    1.0f + (2.0f * (float)n_lw + 2.0f * lg_w + (float)nc * (1.0f / 32.0f) + 40.0f) * kU32;
                // long chains (few lanes per node) are summed in blocks: every
                // kFFRenorm terms the normalised block joins a running total
                // by an accurate double-float add, so the rounding of the low
                // parts no longer accumulates along the whole chain
                const int n_ch = (n_lw + 1) / 2 + 1;
                const bool blocked = n_ch > 16;
                const float c_sb = blocked ? 3.0f * (float)((n_ch + kFFRenorm - 1) / kFFRenorm) +
                                                 3.0f * lg_w + 114.0f
                                           : 9.5f * (float)n_ch + 3.0f * lg_w + 43.0f;
                const float coord_term = (14.7f * xscale + 44.0f) * s_wabs;
                __shared__ float s_pair[2][kGWarps / 2][8];
                for (int it = 0; it < roundsw; ++it) {
                    const int q = p0 + teamw + it * nteamsw;
                    const bool act = q < p1;
                    const int qq = act ? q : p0;
                    // the node's coordinates: high part = the FP32 copy, low part
                    const float4 xh = ldcg(a.xg32 + qq), xlo = ldcg(a.xgl + qq);
                    const float qxh = xh.x, qxl = xlo.x, qyh = xh.y, qyl = xlo.y, qzh = xh.z,
                                qzl = xlo.z;
                    ff fx{0.0f, 0.0f}, fy{0.0f, 0.0f}, fz{0.0f, 0.0f};
                    float sb = 0.0f;
                    // two centres (j, j + ts) per step in paired registers
                    const f2 z2 = f2_pack(0.0f, 0.0f);
                    ff2 gx{z2, z2}, gy{z2, z2}, gz{z2, z2};
                    ff2 tx{z2, z2}, ty{z2, z2}, tz{z2, z2};   // block totals (long chains)
                    const f2 bxh = f2_bcast(qxh), bxl = f2_bcast(qxl), byh = f2_bcast(qyh),
                             byl = f2_bcast(qyl), bzh = f2_bcast(qzh), bzl = f2_bcast(qzl);
                    int j = subw;
                    int nren = 0;
                    for (; j + tsw < nc; j += 2 * tsw) {
                        if (++nren == kFFRenorm) {
                            // error-free renormalisation: the low parts restart
                            // below one ulp of the high parts
                            nren = 0;
                            gx = two_sum2(gx.h, gx.l);
                            gy = two_sum2(gy.h, gy.l);
                            gz = two_sum2(gz.h, gz.l);
                            if (blocked) {
                                tx = ff_add2(tx, gx);
                                ty = ff_add2(ty, gy);
                                tz = ff_add2(tz, gz);
                                gx = ff2{z2, z2};
                                gy = ff2{z2, z2};
                                gz = ff2{z2, z2};
                            }
                        }
                        const int j2 = j + tsw;
                        const float4 ch0 = smem ? cw[j] : ldcg(cw + j);
                        const float4 cl0 = smem ? cw[pst + j] : ldcg(cw + pst + j);
                        const float4 wh0 = smem ? cw[2 * pst + j] : ldcg(cw + 2 * pst + j);
                        const float4 wl0 = smem ? cw[3 * pst + j] : ldcg(cw + 3 * pst + j);
                        const float4 ch1 = smem ? cw[j2] : ldcg(cw + j2);
                        const float4 cl1 = smem ? cw[pst + j2] : ldcg(cw + pst + j2);
                        const float4 wh1 = smem ? cw[2 * pst + j2] : ldcg(cw + 2 * pst + j2);
                        const float4 wl1 = smem ? cw[3 * pst + j2] : ldcg(cw + 3 * pst + j2);
                        const ff2 s2 = dist2_gs2(bxh, bxl, byh, byl, bzh, bzl,
                                                 f2_pack(ch0.x, ch1.x), f2_pack(cl0.x, cl1.x),
                                                 f2_pack(ch0.y, ch1.y), f2_pack(cl0.y, cl1.y),
                                                 f2_pack(ch0.z, ch1.z), f2_pack(cl0.z, cl1.z));
                        const ff2 ph = phi_ff2_s(s2);
                        ff_fma_acc2(gx, f2_pack(wh0.x, wh1.x), f2_pack(wl0.x, wl1.x), ph);
                        ff_fma_acc2(gy, f2_pack(wh0.y, wh1.y), f2_pack(wl0.y, wl1.y), ph);
                        ff_fma_acc2(gz, f2_pack(wh0.z, wh1.z), f2_pack(wl0.z, wl1.z), ph);
                        float p0, p1;
                        f2_unpack(ph.h, p0, p1);
                        sb = fmaf(wh1.w, p1, fmaf(wh0.w, p0, sb));
                    }
                    if (j < nc) {
                        const float4 ch = smem ? cw[j] : ldcg(cw + j);
                        const float4 cl = smem ? cw[pst + j] : ldcg(cw + pst + j);
                        const float4 wh = smem ? cw[2 * pst + j] : ldcg(cw + 2 * pst + j);
                        const float4 wl = smem ? cw[3 * pst + j] : ldcg(cw + 3 * pst + j);
                        const ff s2 = dist2_gs(qxh, qxl, qyh, qyl, qzh, qzl, ch.x, cl.x, ch.y,
                                               cl.y, ch.z, cl.z);
                        const ff ph = phi_ff_s(s2);
                        ff_fma_acc(fx, wh.x, wl.x, ph);
                        ff_fma_acc(fy, wh.y, wl.y, ph);
                        ff_fma_acc(fz, wh.z, wl.z, ph);
                        sb = fmaf(wh.w, ph.h, sb);
                    }
                    // the lane's three accumulators (each an unnormalised
                    // pair) summed and reduced over the team in double-float
                    // on the FP32 pipe
                    auto lane_sum = [&](const ff2 &g, const ff &f) {
                        float h0, h1, l0, l1;
                        f2_unpack(g.h, h0, h1);
                        f2_unpack(g.l, l0, l1);
                        return ff_add(ff_add(two_sum(h0, l0), two_sum(h1, l1)), two_sum(f.h, f.l));
                    };
                    if (blocked) {
                        gx = ff_add2(tx, two_sum2(gx.h, gx.l));
                        gy = ff_add2(ty, two_sum2(gy.h, gy.l));
                        gz = ff_add2(tz, two_sum2(gz.h, gz.l));
                    }
                    ff sx = lane_sum(gx, fx), sy = lane_sum(gy, fy), sz = lane_sum(gz, fz);
                    for (int o = 1; o < min(tsw, 32); o <<= 1) {
                        sx = ff_add(sx, ff{__shfl_xor_sync(0xffffffffu, sx.h, o),
                                           __shfl_xor_sync(0xffffffffu, sx.l, o)});
                        sy = ff_add(sy, ff{__shfl_xor_sync(0xffffffffu, sy.h, o),
                                           __shfl_xor_sync(0xffffffffu, sy.l, o)});
                        sz = ff_add(sz, ff{__shfl_xor_sync(0xffffffffu, sz.h, o),
                                           __shfl_xor_sync(0xffffffffu, sz.l, o)});
                    }
                    sb = team_sum(sb, min(tsw, 32));
                    if (wide) {
                        // the odd warp of the pair hands its sums to the even
                        // one (one more team level); buffers alternate by
                        // round, so one 64-thread barrier per round suffices
                        float *sp = s_pair[it & 1][warp >> 1];
                        if ((warp & 1) && lane == 0) {
                            sp[0] = sx.h;
                            sp[1] = sx.l;
                            sp[2] = sy.h;
                            sp[3] = sy.l;
                            sp[4] = sz.h;
                            sp[5] = sz.l;
                            sp[6] = sb;
                        }
                        asm volatile("bar.sync %0, 64;" ::"r"(1 + (warp >> 1)) : "memory");
                        if (!(warp & 1) && lane == 0) {
                            sx = ff_add(sx, ff{sp[0], sp[1]});
                            sy = ff_add(sy, ff{sp[2], sp[3]});
                            sz = ff_add(sz, ff{sp[4], sp[5]});
                            sb += sp[6];
                        }
                    }
                    if (act && subw == 0 && !ldcg(a.in_s + q)) {
                        const float4 dh = ldcg(a.dgh + q), dl = ldcg(a.dgl + q);
                        const int qnode = ldcg(a.node_of_pos + q);
                        // E = |dr - F| in double-float; FP64 only converts the
                        // result (an FP64 instruction costs a warp ~30x an
                        // FP32 one here)
                        const ff ex = ff_add(ff{dh.x, dl.x}, ff{-sx.h, -sx.l});
                        const ff ey = ff_add(ff{dh.y, dl.y}, ff{-sy.h, -sy.l});
                        const ff ez = ff_add(ff{dh.z, dl.z}, ff{-sz.h, -sz.l});
                        const ff ef = ff_sqrt(ff_add(ff_add(ff_sqr(ex), ff_sqr(ey)), ff_sqr(ez)));
                        const double e = (double)ef.h + (double)ef.l;
                        const float dabs = fabsf(dh.x) + fabsf(dh.y) + fabsf(dh.z);
                        // bound of |E~ - E|: ff rounding of phi, products and
                        // sums (proportional to sum |w| phi + |dr|), of the
                        // coordinate splits (max|x|/R * sum |w|) and of the
                        // square root; the FP32 evaluation of the bound is
                        // rounded up by the factor
                        const float bf =
                            fmaxf(kU32Sq * (c_sb * sb + 4.0f * dabs + coord_term + 50.0f * ef.h) *
                                      b_upw,
                                  1e-18f);
                        a.u32[q] = bf;
                        a.e64[q] = e;
                        const unsigned long long upb = dbits(e + (double)bf);
                        if (look >= 0 && upb > estar_b)
                            first = min(first, (long long)((q - look + nb) % nb));
                        mxb = max(mxb, dbits(e));
                        lsq = fmaf(ef.h, ef.h, lsq);
                        if (argmax) {
                            const unsigned long long k2 = key_f64(e, qnode);
                            if (lead_better(k2, e, key, e_lead)) {
                                key = k2;
                                e_lead = e;
                                b_lead = (double)bf;
                                p_lead = q;
                            }
                        }
                        if (upb > u1) {
                            u2 = u1;
                            u1 = upb;
                            n1 = qnode;
                        } else if (upb > u2) {
                            u2 = upb;
                        }
                    }
                }
                if (g_vb == 0 && tid == 0)
                    pairsff += (long long)nq * nc;
            }
        }
        // ---- reductions, one record per CTA: the leader (largest key) with its
        // error, bound and position; the maximum and the sum of squares of E;
        // the two largest upper bounds and the node of the largest.  Only the
        // first lane of each team holds data, so warps combine lanes at
        // distances >= ts; warp 0 combines the warps; after the barrier warp 0
        // of every CTA combines the G records in the same order.
        phase(9);
        {
            auto merge = [](unsigned long long &k, double &el, double &bl, long long &pl,
                            unsigned long long &v1, unsigned long long &v2, long long &m1,
                            unsigned long long &mx, float &sq, long long &fr,
                            unsigned long long ok_, double oel, double obl, long long opl,
                            unsigned long long ov1, unsigned long long ov2, long long om1,
                            unsigned long long omx, float osq, long long ofr) {
                fr = min(fr, ofr);
                if (lead_better(ok_, oel, k, el)) {
                    k = ok_;
                    el = oel;
                    bl = obl;
                    pl = opl;
                }
                if (ov1 > v1 || (ov1 == v1 && om1 >= 0 && (m1 < 0 || om1 < m1))) {
                    v2 = max(v1, ov2);
                    v1 = ov1;
                    m1 = om1;
                } else {
                    v2 = max(v2, ov1);
                }
                mx = max(mx, omx);
                sq += osq;
            };
            for (int o = 16; o >= ts; o >>= 1) {
                const unsigned long long ok_ = __shfl_xor_sync(0xffffffffu, key, o);
                const double oel = __shfl_xor_sync(0xffffffffu, e_lead, o);
                const double obl = __shfl_xor_sync(0xffffffffu, b_lead, o);
                const long long opl = __shfl_xor_sync(0xffffffffu, p_lead, o);
                const unsigned long long ov1 = __shfl_xor_sync(0xffffffffu, u1, o);
                const unsigned long long ov2 = __shfl_xor_sync(0xffffffffu, u2, o);
                const long long om1 = __shfl_xor_sync(0xffffffffu, n1, o);
                const unsigned long long omx = __shfl_xor_sync(0xffffffffu, mxb, o);
                const float osq = __shfl_xor_sync(0xffffffffu, lsq, o);
                const long long ofr = __shfl_xor_sync(0xffffffffu, first, o);
                merge(key, e_lead, b_lead, p_lead, u1, u2, n1, mxb, lsq, first, ok_, oel, obl,
                      opl, ov1, ov2, om1, omx, osq, ofr);
            }
            __shared__ EvalRec s_rec[kGWarps];
            if (lane == 0)
                s_rec[warp] = EvalRec{mxb, u1, u2, e_lead, b_lead, lsq, 0,
                                      n1, (long long)key, p_lead, first};
            __syncthreads();
            if (warp == 0) {
                EvalRec t = lane < kGWarps ? s_rec[lane] : kEmptyRec;
                unsigned long long k = (unsigned long long)t.key;
                for (int o = kGWarps / 2; o > 0; o >>= 1) {
                    const unsigned long long ok_ = __shfl_xor_sync(0xffffffffu, k, o);
                    const double oel = __shfl_xor_sync(0xffffffffu, t.e_lead, o);
                    const double obl = __shfl_xor_sync(0xffffffffu, t.b_lead, o);
                    const long long opl = __shfl_xor_sync(0xffffffffu, t.p_lead, o);
                    const unsigned long long ov1 = __shfl_xor_sync(0xffffffffu, t.u1, o);
                    const unsigned long long ov2 = __shfl_xor_sync(0xffffffffu, t.u2, o);
                    const long long om1 = __shfl_xor_sync(0xffffffffu, t.n1, o);
                    const unsigned long long omx = __shfl_xor_sync(0xffffffffu, t.mx, o);
                    const float osq = __shfl_xor_sync(0xffffffffu, t.sq, o);
                    const long long ofr = __shfl_xor_sync(0xffffffffu, t.first, o);
                    merge(k, t.e_lead, t.b_lead, t.p_lead, t.u1, t.u2, t.n1, t.mx, t.sq, t.first,
                          ok_, oel, obl, opl, ov1, ov2, om1, omx, osq, ofr);
                }
                t.key = (long long)k;
                if (lane == 0)
                    a.rec[(size_t)(use & 1) * kMaxGrid + g_vb] = t;
            }
        }
        phase(10);
        GSYNC_B();
        double gu1 = 0.0, gu2 = 0.0;
        long long gn1 = -1;
        {
            __shared__ EvalRec s_g;
            if (warp == 0) {
                EvalRec t = kEmptyRec;
                unsigned long long k = 0;
                const EvalRec *rb = a.rec + (size_t)(use & 1) * kMaxGrid;
                auto merge = [](unsigned long long &k, EvalRec &t, const EvalRec &o) {
                    if (lead_better((unsigned long long)o.key, o.e_lead, k, t.e_lead)) {
                        k = (unsigned long long)o.key;
                        t.e_lead = o.e_lead;
                        t.b_lead = o.b_lead;
                        t.p_lead = o.p_lead;
                    }
                    if (o.u1 > t.u1 || (o.u1 == t.u1 && o.n1 >= 0 && (t.n1 < 0 || o.n1 < t.n1))) {
                        t.u2 = max(t.u1, o.u2);
                        t.u1 = o.u1;
                        t.n1 = o.n1;
                    } else {
                        t.u2 = max(t.u2, o.u1);
                    }
                    t.mx = max(t.mx, o.mx);
                    t.sq += o.sq;
                    t.first = min(t.first, o.first);
                };
                for (int b = lane; b < G; b += 32) {
                    const longlong2 *src = (const longlong2 *)(rb + b);
                    const longlong2 w0 = __ldcg(src), w1 = __ldcg(src + 1), w2 = __ldcg(src + 2),
                                    w3 = __ldcg(src + 3), w4 = __ldcg(src + 4);
                    EvalRec o;
                    o.mx = (unsigned long long)w0.x;
                    o.u1 = (unsigned long long)w0.y;
                    o.u2 = (unsigned long long)w1.x;
                    o.e_lead = __longlong_as_double(w1.y);
                    o.b_lead = __longlong_as_double(w2.x);
                    o.sq = __int_as_float((int)(w2.y & 0xffffffffll));
                    o.pad = 0;
                    o.n1 = w3.x;
                    o.key = w3.y;
                    o.p_lead = w4.x;
                    o.first = w4.y;
                    merge(k, t, o);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    EvalRec q;
                    q.key = (long long)__shfl_xor_sync(0xffffffffu, k, o);
                    q.e_lead = __shfl_xor_sync(0xffffffffu, t.e_lead, o);
                    q.b_lead = __shfl_xor_sync(0xffffffffu, t.b_lead, o);
                    q.p_lead = __shfl_xor_sync(0xffffffffu, t.p_lead, o);
                    q.u1 = __shfl_xor_sync(0xffffffffu, t.u1, o);
                    q.u2 = __shfl_xor_sync(0xffffffffu, t.u2, o);
                    q.n1 = __shfl_xor_sync(0xffffffffu, t.n1, o);
                    q.mx = __shfl_xor_sync(0xffffffffu, t.mx, o);
                    q.sq = __shfl_xor_sync(0xffffffffu, t.sq, o);
                    q.first = __shfl_xor_sync(0xffffffffu, t.first, o);
                    merge(k, t, q);
                }
                t.key = (long long)k;
                if (lane == 0)
                    s_g = t;
            }
            __syncthreads();
            out.key = (unsigned long long)s_g.key;
            out.gmax = bitsd(s_g.mx);
            out.gsq = (double)s_g.sq;
            out.e_lead = s_g.e_lead;
            out.b_lead = s_g.b_lead;
            out.p_lead = (int)s_g.p_lead;
            out.first = s_g.first;
            gu1 = bitsd(s_g.u1);
            gu2 = bitsd(s_g.u2);
            gn1 = s_g.n1;
            // screened modes: the certified maximum is the largest upper
            // bound E~ + beta (E~ alone may overstate or understate E)
            if (screened)
                out.gmax = gu1;
            __syncthreads();
            ++use;
        }
        phase(1);
        ++ev;
        if (screened && argmax && out.key) {
            // ---- certification from the bounds: the leader b (largest E~)
            // is the argmax when E~_b - beta_b exceeds every other node's
            // upper bound; the E > E* decision is certified when the bound
            // interval of the leader lies on one side of E*.
            const int nb_ = key_node(out.key);
            const double lower = out.e_lead - out.b_lead;
            const double other = (gn1 == nb_) ? gu2 : gu1;
            // certified: every node is <= E* (no append whoever leads), or
            // the leader is the unique maximum and lies above E*
            const bool none_above = gu1 <= estar;
            const bool lead_adds = lower > other && lower > estar;
            if (!(none_above || lead_adds)) {
                // ---- pass 2 (rare): FP64 re-score of every node whose upper
                // bound reaches the leader's lower bound
                phase(2);
                double bv = -1.0;   // exact (value, node) argmax of the re-scored nodes
                long long bi = -1;
                const double thr = lower;   // the maximum is >= the leader's lower bound
                for (int it = 0; it < rounds; ++it) {
                    const int q = p0 + team + it * nteams;
                    const bool act = q < p1;
                    bool need = false;
                    if (act && !ldcg(a.in_s + q))
                        need = ldcg(a.e64 + q) + (double)ldcg(a.u32 + q) >= thr;
                    if (__ballot_sync(0xffffffffu, need) == 0u)
                        continue;
                    const double e = team_error_f64(a, act ? q : p0, nc, sub, ts);
                    if (need && sub == 0) {
                        ++rescored_local;
                        a.e64[q] = e;
                        a.u32[q] = 0.0f;
                        pick(bv, bi, e, (long long)ldcg(a.node_of_pos + q));
                    }
                }
                block_pick(red, bv, bi);
                if (tid == 0) {
                    part(use)[g_vb] = bv;
                    parti(use)[g_vb] = bi;
                }
                GSYNC_B();
                double gv;
                long long gi;
                grid_pick_reduce(part(use), parti(use), G, gv, gi);
                ++use;
                if (gi >= 0) {
                    out.key = key_f64(gv, (int)gi);
                    out.p_lead = ldcg(a.pos_of_node + gi);
                    out.e_lead = gv;
                    out.b_lead = 0.0;
                    // every node left out has E < thr <= the leader's E, so
                    // the largest FP64 value among the re-scored nodes is the
                    // maximum
                    out.gmax = gv;
                }
            }
        }
        phase(5);
        return true;
    };

    // ---------------- main loop (k counts iterations from 3) ---------------
    // Stops after m consecutive iterations without an append: those m groups
    // cover every node (Sec. 3) and were evaluated with the same weights, so
    // the largest of their maxima is the certified global maximum.
    long long k = 3, nhist = 0, nfull = 0, idle = 0;
    double run_max = 0.0, run_sq = 0.0;
    int status = RBF_OK;
    const bool hist_full = a.hist != nullptr && (a.flags & RBF_FLAG_HISTORY_FULL) != 0;
    // groups of the iterations before scan_end_k were scanned by a look-ahead
    // with the current weights (their errors and bounds are in e64/u32); an
    // append clears it
    long long scan_end_k = 0;
    for (;; ++k) {
        const int gi = (int)(k % m);
        const int g0 = goff(gi, nb, m), g1 = goff(gi + 1, nb, m);
        EvalOut eo;
        if (!evaluate(g0, g1, true, false, eo, -1, false))
            return;
        int add_node = -1, add_pos = -1;
        double eloc = -1.0;
        if (eo.key) {
            add_node = key_node(eo.key);
            add_pos = eo.p_lead;
            eloc = eo.e_lead;
            if (!(eloc > estar))
                add_node = -1;
        }
        // peak selection: several separated nodes of this group at once
        __shared__ int s_pk_pos[kMaxPeaks], s_pk_node[kMaxPeaks];
        __shared__ D4 s_pk_x[kMaxPeaks];
        __shared__ float4 s_pk_h[kMaxPeaks], s_pk_l[kMaxPeaks];
        int n_add = add_node >= 0 ? 1 : 0;
        // (an iteration whose certified maximum is <= E* has no candidate)
        if (kPeaks && a.peaks > 1 && add_node >= 0) {
            const bool screened = a.prec != RBF_PREC_F64;
            int c = select_peaks(a, g0, g1, estar, !screened, xscale, use, epoch, s_pk_pos,
                                 s_pk_node, s_pk_x, s_pk_h, s_pk_l);
            if (c == -2)
                return;
            if (c < 0) {
                // the bounds did not certify the selection: every candidate
                // of the group in FP64, then the selection on exact values
                phase(2);
                const int nq = g1 - g0, ts = team_size(nq, G), sub = lane & (ts - 1);
                const int team = gtid / ts, nteams = gthreads / ts;
                const int rounds = (nq + nteams - 1) / nteams;
                for (int it = 0; it < rounds; ++it) {
                    const int q = g0 + team + it * nteams;
                    const bool act = q < g1;
                    bool need = false;
                    if (act && !ldcg(a.in_s + q)) {
                        const float b = ldcg(a.u32 + q);
                        need = b > 0.0f && ldcg(a.e64 + q) + (double)b > estar;
                    }
                    if (__ballot_sync(0xffffffffu, need) == 0u)
                        continue;
                    const double e = team_error_f64(a, act ? q : g0, nc, sub, ts);
                    if (need && sub == 0) {
                        a.e64[q] = e;
                        a.u32[q] = 0.0f;
                        ++rescored_local;
                    }
                }
                GSYNC();
                c = select_peaks(a, g0, g1, estar, true, xscale, use, epoch, s_pk_pos, s_pk_node,
                                 s_pk_x, s_pk_h, s_pk_l);
                if (c == -2)
                    return;
                phase(5);
            }
            n_add = c;
            add_node = n_add > 0 ? s_pk_node[0] : -1;
        }
        const long long nc_before = nc;
        if (add_node >= 0) {
            bool failed = false;
            if (kPeaks && a.peaks > 1 && n_add > 1 && a.nc_max - nc >= 2) {
                // several peaks: one block append
                const int kb = min(n_add, a.nc_max - nc);
                phase(3);
                const int ar = chol_append_block(a, nc, min_piv, kb, s_pk_pos, s_pk_node, k,
                                                 epoch);
                phase(5);
                if (ar != kAppendOk) {
                    status = RBF_E_NOT_SPD;   // or the latched timeout, which wins
                    failed = true;
                } else if (kb < n_add) {
                    status = RBF_E_NC_MAX;
                    failed = true;
                }
            } else {
                for (int r = 0; r < n_add; ++r) {
                    if (nc >= a.nc_max) {
                        status = RBF_E_NC_MAX;
                        failed = true;
                        break;
                    }
                    phase(3);
                    const int ar = kPeaks && a.peaks > 1
                                       ? chol_append(a, red, nc, use, min_piv, s_pk_pos[r],
                                                     s_pk_node[r], k, epoch, bscratch())
                                       : chol_append(a, red, nc, use, min_piv, add_pos, add_node,
                                                     k, epoch, bscratch());
                    staged_nc = -1;
                    phase(5);
                    if (ar != kAppendOk) {
                        status = RBF_E_NOT_SPD;   // or the latched timeout, which wins
                        failed = true;
                        break;
                    }
                }
            }
            if (failed)
                break;
            idle = 0;
            run_max = 0.0;
            run_sq = 0.0;
            scan_end_k = 0;
        } else {
            ++idle;
            run_max = fmax(run_max, eo.gmax);
            run_sq += eo.gsq;
        }
        double gmax = -1.0, grms = -1.0;
        if (hist_full && ((k - 2) % m) == 0) {
            EvalOut d;
            if (!evaluate(0, nb, false, true, d, -1, false))
                return;
            ++nfull;
            gmax = d.gmax;
            grms = sqrt(d.gsq / (double)nb);
        }
        if (g_vb == 0 && tid == 0 && a.hist && nhist < a.hist_cap) {
            double *h = a.hist + RBF_HIST_COLS * nhist;
            h[0] = (double)k;
            h[1] = (double)nc_before;
            h[2] = eloc;
            h[3] = gmax;
            h[4] = grms;
            h[5] = (double)add_node;
        }
        ++nhist;
        if (idle >= m)
            break;
        // Look-ahead: after kLookIdle iterations without an append, evaluate
        // every node once with the unchanged weights.  Groups whose nodes are
        // all certified <= E* would add nothing when their turn comes, so the
        // literal sequence continues at the first group (in cyclic order
        // from the next one) that holds a node possibly above E*; with none,
        // the run ends where m idle iterations would end it.  A later
        // look-ahead of the same idle run (a flagged group whose nodes all
        // turned out <= E*) only scans the stored errors and bounds.
        // Look-ahead over an idle run: the weights cannot change until the
        // next append, so the groups still to come are scanned in chunks of
        // kLookChunk groups, in their cyclic order, with the current weights,
        // up to the first group holding a node possibly above E* (upper bound
        // E~ + beta > E*); the iterations before it would add nothing and are
        // certified without their own evaluation.  With none before the run
        // would end (m idle iterations), it ends here.  Chunks scanned earlier
        // in the same idle run are read back from the stored errors.  A
        // scan pays only when one group's pairs cost at most half an idle
        // iteration (a deterministic model, so every CTA decides alike).
        const double look_rate = a.prec == RBF_PREC_F32X2 ? kLookPairsFF
                                 : a.prec == RBF_PREC_F32 ? kLookPairsF32
                                                          : kLookPairsF64;
        const bool look_pays =
            (double)((nb + m - 1) / m) * (double)nc <= 0.5 * look_rate * G;
        if (idle >= kLookIdle && m > 2 * kLookIdle && !hist_full && look_pays) {
            const long long k_last = k + (m - idle);   // the literal run's last iteration
            long long ks = k + 1, found = -1;
            bool fresh = false;
            // chunks while ks <= k_last; then, with no candidate, one pass over
            // the stored errors of every node (each group was evaluated or
            // scanned with these weights in this idle run) for the run's
            // certified maximum and RMS.  One call site keeps the kernel small.
            for (;;) {
                const bool final_pass = ks > k_last;
                const int g0 = final_pass ? 0 : (int)(ks % m);
                const bool cached = final_pass || ks < scan_end_k;
                long long ke = min(ks + (long long)kLookChunk, k_last + 1);
                ke = min(ke, ks + (long long)(m - g0));   // no wrap inside a chunk
                if (cached && !final_pass)
                    ke = min(ke, scan_end_k);
                const int p0 = final_pass ? 0 : goff(g0, nb, m);
                const int p1 = final_pass ? nb : goff(g0 + (int)(ke - ks), nb, m);
                EvalOut la;
                if (!evaluate(p0, p1, false, false, la, p0, cached))
                    return;
                if (final_pass) {
                    run_max = la.gmax;
                    run_sq = la.gsq;
                    break;
                }
                if (!cached) {
                    scan_end_k = ke;
                    fresh = true;
                }
                if (la.first != kNoRank) {
                    const int pos = p0 + (int)la.first;
                    const int base = nb / m, rem = nb % m;
                    const int g = pos < rem * (base + 1) ? pos / (base + 1)
                                                         : rem + (pos - rem * (base + 1)) / base;
                    found = ks + (g - g0);
                    break;
                }
                ks = ke;
            }
            if (fresh)
                ++nfull;
            // idle iterations certified without evaluation
            const long long skip = found >= 0 ? found - (k + 1) : m - idle;
            if (g_vb == 0 && tid == 0 && a.hist)
                for (long long s2 = 1; s2 <= skip && nhist + s2 - 1 < a.hist_cap; ++s2) {
                    double *h = a.hist + RBF_HIST_COLS * (nhist + s2 - 1);
                    h[0] = (double)(k + s2);
                    h[1] = (double)nc;
                    h[2] = -1.0;
                    h[3] = -1.0;
                    h[4] = -1.0;
                    h[5] = -1.0;
                }
            k += skip;
            idle += skip;
            nhist += skip;
            if (idle >= m)
                break;
        }
    }
    // final weights of the selected set (row a9): FP64 refinement with Z
    double maxres = -1.0;
    phase(4);
    if (a.w_out && nc > 0) {
        if (!refine_weights(a, red, nc, use, epoch, a.refine_steps, a.spos, a.rvec, a.tvec,
                            maxres))
            return;
        for (int j = gtid; j < nc; j += gthreads) {
            const D4 w = ldcg(a.w64 + j);
            a.w_out[3 * j] = w.x;
            a.w_out[3 * j + 1] = w.y;
            a.w_out[3 * j + 2] = w.z;
        }
    }
    phase(5);
    if (g_vb == 0 && tid == 0) {
        if (a.nc_out)
            *a.nc_out = nc;
        for (int i = 0; i < 12; ++i)
            ctl->phase_ns[i] = ph_acc[i];
        ctl->phase_ns[6] = g_bar_wait_ns;
        if (status != RBF_OK)
            atomicCAS(&ctl->status, (int)RBF_OK, status);
        ctl->max_resid = maxres;
        ctl->barriers = (long long)epoch + bar_extra;
        ctl->estar = estar;
        ctl->nc = nc;
        ctl->iterations = k - 3 + 1;
        ctl->full_checks = nfull;
        ctl->pairs_f32 = pairs32;
        ctl->pairs_f64 = pairs64;
        ctl->pairs_ff = pairsff;
        ctl->final_max = idle >= m ? run_max : -1.0;
        ctl->final_rms = idle >= m ? sqrt(run_sq / (double)nb) : -1.0;
        ctl->min_pivot = min_piv;
        ctl->n_hist = nhist;
    }
    if (rescored_local)
        atomicAdd(&ctl->rescored, rescored_local);
#undef GSYNC
#undef GSYNC_B
}

// One problem on the whole grid.
__global__ void __launch_bounds__(kGThreads, 1) k_greedy(GreedyArgs a)
{
    if (threadIdx.x == 0) {
        g_vb = blockIdx.x;
        g_vg = gridDim.x;
    }
    __syncthreads();
    greedy_body<false>(a);
}

// The peak-selection variant (several separated nodes per iteration).
__global__ void __launch_bounds__(kGThreads, 1) k_greedy_peaks(GreedyArgs a)
{
    if (threadIdx.x == 0) {
        g_vb = blockIdx.x;
        g_vg = gridDim.x;
    }
    __syncthreads();
    greedy_body<true>(a);
}

// Many problems in one launch: problem i runs on CTAs [cta_start[i],
// cta_start[i + 1]) with its own workspace, control block and barrier.
__global__ void __launch_bounds__(kGThreads, 2)
k_greedy_batched(const GreedyArgs *__restrict__ args, const int *__restrict__ cta_start, int B)
{
    __shared__ int s_prob;
    if (threadIdx.x == 0) {
        int lo = 0, hi = B - 1;   // last i with cta_start[i] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (cta_start[mid] <= (int)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_prob = lo;
        g_vb = blockIdx.x - cta_start[lo];
        g_vg = cta_start[lo + 1] - cta_start[lo];
    }
    __syncthreads();
    const GreedyArgs a = args[s_prob];
    greedy_body<false>(a);
}


// ---------------------------------------------------------------------------
// Support weights (Eqs. 4-5 on S): recurrence-Cholesky appends in the given
// order, then FP64 iterative refinement W += Z^T Z (dX_S - Phi_SS W) with the
// residual recomputed from coordinates.  One cooperative launch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads, 1)
k_solve(GreedyArgs a, const int32_t *__restrict__ sel, int nc_total, int steps,
        D4 *__restrict__ rvec, D4 *__restrict__ tvec, double *__restrict__ w_out,
        const double *__restrict__ rhs, int reuse)
{
    __shared__ Red red;
    if (threadIdx.x == 0) {
        g_vb = blockIdx.x;
        g_vg = gridDim.x;
        g_bar = &a.ctl->bar;
    }
    __syncthreads();
    GreedyCtl *ctl = a.ctl;
    const int G = g_vg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtid = g_vb * kGThreads + tid;
    const int gthreads = G * kGThreads;
    int use = 0;
    unsigned int epoch = 0;
    auto part = [&](int u) { return a.part + (size_t)(u & 1) * kMaxGrid * 4; };
#define GSYNC()                                                                   \
    do {                                                                          \
        if (!grid_barrier(g_bar, &ctl->status, (unsigned)G, a.barrier_ns, epoch, (unsigned)g_vb)) \
            return;                                                               \
    } while (0)

    // a fresh factorisation passes three barriers per support node: place
    // the barrier first (a reused factor only refines, and keeps the
    // control block's barrier)
    long long bar_extra = 0;
    if (!reuse && !place_barrier(a, G, epoch, bar_extra))
        return;
    double bad = 0.0;
    for (int j = gtid; j < nc_total; j += gthreads) {
        const int node = sel[j];
        if (node < 0 || node >= a.nb) {
            bad = fmax(bad, 2.0);
            continue;
        }
        const double x = a.xb[3 * node] * a.inv_r, y = a.xb[3 * node + 1] * a.inv_r,
                     z = a.xb[3 * node + 2] * a.inv_r;
        // right-hand side: the prescribed displacements dX_S, or a caller's
        // nc x 3 array (support order)
        const double *rr = rhs ? rhs + 3 * j : a.db + 3 * node;
        const double d0 = rr[0], d1 = rr[1], d2 = rr[2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(d0) || !isfinite(d1) ||
            !isfinite(d2))
            bad = fmax(bad, 1.0);
        a.xg64[j] = mk4(x, y, z, 0.0);
        a.dg64[j] = mk4(d0, d1, d2, 0.0);
        a.in_s[j] = 0;
    }
    {
        double mx = bad;
        for (int o = 16; o > 0; o >>= 1)
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        __syncthreads();
        if (lane == 0)
            red.v[warp] = mx;
        __syncthreads();
        if (tid == 0) {
            for (int k = 1; k < kGWarps; ++k)
                mx = fmax(mx, red.v[k]);
            part(use)[4 * g_vb] = mx;
        }
    }
    GSYNC();
    {
        double g4[4];
        grid_max4(part(use), G, g4);   // slot 0 of each CTA's partial
        ++use;
        if (g4[0] > 0.0) {
            if (g_vb == 0 && tid == 0)
                ctl->status = g4[0] > 1.5 ? RBF_E_ARG : RBF_E_NONFINITE;
            return;
        }
    }
    int nc = 0;
    double min_piv = INFINITY;
    if (reuse) {
        // the factor Z = L^-1 and the centres of an earlier launch on the same
        // workspace and support set: start from W = 0, so the first
        // refinement step is the solve W = Z^T Z rhs
        for (int j = gtid; j < nc_total; j += gthreads)
            a.w64[j] = mk4(0.0, 0.0, 0.0, 0.0);
        nc = nc_total;
        ++steps;
        GSYNC();
    }
    for (int j = nc; j < nc_total; ++j) {
        const int node = sel[j];
        const int r = chol_append(a, red, nc, use, min_piv, j, node, -1, epoch);
        if (r != kAppendOk) {
            if (g_vb == 0 && tid == 0) {
                ctl->nc = nc;
                ctl->min_pivot = min_piv;
            }
            return;
        }
    }
    double maxres = 0.0;
    if (!refine_weights(a, red, nc, use, epoch, steps, nullptr, rvec, tvec, maxres))
        return;
    for (int j = gtid; j < nc; j += gthreads) {
        const D4 w = ldcg(a.w64 + j);
        w_out[3 * j] = w.x;
        w_out[3 * j + 1] = w.y;
        w_out[3 * j + 2] = w.z;
    }
    if (g_vb == 0 && tid == 0) {
        ctl->nc = nc;
        ctl->min_pivot = min_piv;
        ctl->final_max = maxres;
    }
#undef GSYNC
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
struct GreedyWs {
    size_t ctl, part, parti, perm, node_of_pos, pos_of_node, xg64, dg64, xg32, xgl, dgh, dgl,
        in_s, u32, e64,
        spos, c64, w64, cw32, cwff, y64, z, zt, bvec, lvec, rvec, tvec, rec, bmat, lmat, cmat,
        bpart, total;
};

static GreedyWs greedy_ws_layout(int64_t nb, int64_t ncm)
{
    GreedyWs L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.ctl = take(sizeof(GreedyCtl));
    L.part = take(sizeof(double) * 2 * kMaxGrid * 4);
    L.parti = take(sizeof(long long) * 2 * kMaxGrid);
    L.perm = take(sizeof(int32_t) * nb);
    L.node_of_pos = take(sizeof(int32_t) * nb);
    L.pos_of_node = take(sizeof(int32_t) * nb);
    L.xg64 = take(sizeof(D4) * nb);
    L.dg64 = take(sizeof(D4) * nb);
    L.xg32 = take(sizeof(float4) * nb);
    L.xgl = take(sizeof(float4) * nb);
    L.dgh = take(sizeof(float4) * nb);
    L.dgl = take(sizeof(float4) * nb);
    L.in_s = take(nb);
    L.u32 = take(sizeof(float) * nb);
    L.e64 = take(sizeof(double) * nb);
    L.spos = take(sizeof(int32_t) * ncm);
    L.c64 = take(sizeof(D4) * ncm);
    L.w64 = take(sizeof(D4) * ncm);
    L.cw32 = take(sizeof(float4) * 2 * ncm);
    L.cwff = take(sizeof(float4) * 4 * ncm);
    L.y64 = take(sizeof(D4) * ncm);
    L.z = take(sizeof(double) * ncm * ncm);
    L.zt = take(sizeof(double) * ncm * ncm);
    L.bvec = take(sizeof(double) * ncm);
    L.lvec = take(sizeof(double) * ncm);
    L.rvec = take(sizeof(D4) * ncm);
    L.tvec = take(sizeof(D4) * ncm);
    L.rec = take(sizeof(EvalRec) * 2 * kMaxGrid);
    L.bmat = take(sizeof(double) * kMaxPeaks * ncm);
    L.lmat = take(sizeof(double) * kMaxPeaks * ncm);
    L.cmat = take(sizeof(double) * kMaxPeaks * kMaxPeaks);
    L.bpart = take(sizeof(double) * kPeakGrid * kBlkV);
    L.total = o;
    return L;
}

static bool greedy_args_ok(int64_t nb, const rbf_params *p)
{
    return p && nb >= 3 && nb < kMaxNodes && p->m >= 1 && p->m <= nb && p->nc_max >= 3 &&
           p->nc_max <= nb && p->nc_max <= 46340 && p->radius > 0.0 &&
           std::isfinite(p->radius) && p->tol >= 0.0 && std::isfinite(p->tol) &&
           (p->tol_mode == 0 || p->tol_mode == 1) &&
           (p->eval_prec == RBF_PREC_F32 || p->eval_prec == RBF_PREC_F64 ||
            p->eval_prec == RBF_PREC_F32X2) &&
           (p->flags & ~(RBF_FLAG_HISTORY_FULL | RBF_FLAG_TEST_BARRIER_TIMEOUT)) == 0 &&
           p->ctas >= 0;
}

}  // namespace rbf

namespace rbf {
struct SolveWs {
    GreedyWs g;
    size_t sel, rvec, tvec, total;
};

static SolveWs solve_ws_layout(int64_t nc)
{
    SolveWs L{};
    L.g = greedy_ws_layout(nc, nc);
    size_t o = L.g.total;
    L.sel = o;
    o = align_up(o + sizeof(int32_t) * nc, 256);
    L.rvec = o;
    o = align_up(o + sizeof(D4) * nc, 256);
    L.tvec = o;
    o = align_up(o + sizeof(D4) * nc, 256);
    L.total = o;
    return L;
}

static void fill_args(GreedyArgs &a, char *ws, const GreedyWs &L)
{
    a.ctl = (GreedyCtl *)(ws + L.ctl);
    a.perm = (const int32_t *)(ws + L.perm);
    a.node_of_pos = (int32_t *)(ws + L.node_of_pos);
    a.pos_of_node = (int32_t *)(ws + L.pos_of_node);
    a.xg64 = (D4 *)(ws + L.xg64);
    a.dg64 = (D4 *)(ws + L.dg64);
    a.xg32 = (float4 *)(ws + L.xg32);
    a.xgl = (float4 *)(ws + L.xgl);
    a.dgh = (float4 *)(ws + L.dgh);
    a.dgl = (float4 *)(ws + L.dgl);
    a.in_s = (uint8_t *)(ws + L.in_s);
    a.u32 = (float *)(ws + L.u32);
    a.e64 = (double *)(ws + L.e64);
    a.part = (double *)(ws + L.part);
    a.parti = (long long *)(ws + L.parti);
    a.spos = (int32_t *)(ws + L.spos);
    a.c64 = (D4 *)(ws + L.c64);
    a.w64 = (D4 *)(ws + L.w64);
    a.cw32 = (float4 *)(ws + L.cw32);
    a.cwff = (float4 *)(ws + L.cwff);
    a.y64 = (D4 *)(ws + L.y64);
    a.z = (double *)(ws + L.z);
    a.zt = (double *)(ws + L.zt);
    a.bvec = (double *)(ws + L.bvec);
    a.lvec = (double *)(ws + L.lvec);
    a.rvec = (D4 *)(ws + L.rvec);
    a.tvec = (D4 *)(ws + L.tvec);
    a.rec = (EvalRec *)(ws + L.rec);
    a.bmat = (double *)(ws + L.bmat);
    a.lmat = (double *)(ws + L.lmat);
    a.cmat = (double *)(ws + L.cmat);
    a.bpart = (double *)(ws + L.bpart);
}
}  // namespace rbf

using namespace rbf;

extern "C" size_t rbf_greedy_workspace_bytes(int64_t nb, const rbf_params *p)
{
    if (!greedy_args_ok(nb, p))
        return 0;
    return greedy_ws_layout(nb, p->nc_max).total;
}

static rbf_status greedy_launch(const double *d_xb, const double *d_db, int64_t nb,
                                const rbf_params *p, int32_t *d_sel_idx, int64_t *d_sel_iter,
                                double *d_w, double *d_hist, int64_t hist_cap, int64_t *h_nc,
                                int64_t *h_n_hist, rbf_greedy_stats *h_stats, void *d_ws,
                                size_t ws_bytes, void *stream, int peaks, double separation)
{
    if (!greedy_args_ok(nb, p) || !d_xb || !d_db || !d_sel_idx || !h_nc || hist_cap < 0 ||
        (hist_cap > 0 && !d_hist) || p->refine_steps < 0 || p->refine_steps > 16 ||
        peaks < 1 || peaks > kMaxPeaks || !(separation >= 0.0) || !std::isfinite(separation))
        return RBF_E_ARG;
    const GreedyWs L = greedy_ws_layout(nb, p->nc_max);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev) || !dev.coop)
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;

    // the random partition (host, O(N_b)) -- overlaps nothing yet
    std::vector<int32_t> perm((size_t)nb);
    fisher_yates(nb, p->seed, perm.data());
    if (cudaMemsetAsync(ws + L.ctl, 0, sizeof(GreedyCtl), st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.perm, perm.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return RBF_E_CUDA;

    GreedyArgs a{};
    a.xb = d_xb;
    a.db = d_db;
    a.nb = (int)nb;
    a.m = (int)p->m;
    a.nc_max = (int)p->nc_max;
    a.prec = p->eval_prec;
    a.inv_r = 1.0 / p->radius;
    a.tol = p->tol;
    a.tol_mode = p->tol_mode;
    a.flags = p->flags;
    a.barrier_ns = (p->flags & RBF_FLAG_TEST_BARRIER_TIMEOUT) ? 50000000ull : kBarrierLimitNs;
    a.ld = (int)p->nc_max;
    a.sel_idx = d_sel_idx;
    a.sel_iter = d_sel_iter;
    a.hist = hist_cap > 0 ? d_hist : nullptr;
    a.hist_cap = hist_cap;
    a.w_out = d_w;
    a.refine_steps = p->refine_steps;
    a.peaks = peaks;
    a.sep2 = (separation / p->radius) * (separation / p->radius);
    fill_args(a, ws, L);

    // the evaluation table of as many centres as fit beside the kernel's
    // static shared memory (one CTA per SM): about 3,500 double-float or
    // 7,000 FP32 centres on this GPU
    const size_t per_centre = p->eval_prec == RBF_PREC_F32     ? sizeof(float4) * 2
                              : p->eval_prec == RBF_PREC_F32X2 ? sizeof(float4) * 4
                                                               : 0;
    const void *kfn = peaks > 1 ? (const void *)k_greedy_peaks : (const void *)k_greedy;
    cudaFuncAttributes fattr{};
    if (cudaFuncGetAttributes(&fattr, kfn) != cudaSuccess)
        return RBF_E_CUDA;
    const size_t room = dev.smem_optin > fattr.sharedSizeBytes + 1024
                            ? dev.smem_optin - fattr.sharedSizeBytes - 1024 : 0;
    a.smem_cap = per_centre ? (int)std::min<int64_t>(p->nc_max, (int64_t)(room / per_centre)) : 0;
    const size_t smem = per_centre * (size_t)a.smem_cap;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max<size_t>(smem, 1)) != cudaSuccess)
        return RBF_E_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kGThreads, smem) !=
            cudaSuccess ||
        occ < 1)
        return RBF_E_CUDA;
    // grid: enough CTAs for one 32-lane team per node of the largest group,
    // at least 64 (the appends and look-aheads spread their work over the
    // CTAs, and a grid barrier costs about the same at 32 and 64 CTAs), at
    // most one per SM (beyond that every barrier and grid reduction slows
    // more than the evaluation speeds up); p->ctas > 0 overrides (tuning)
    const int64_t gsize = (nb + p->m - 1) / p->m;
    const int64_t want = std::max<int64_t>(64, (gsize * 32 + kGThreads - 1) / kGThreads);
    int grid = (int)std::min<int64_t>(want, (int64_t)dev.sms);
    if (p->ctas > 0)
        grid = std::min(p->ctas, dev.sms * std::min(occ, 2));
    grid = std::min(grid, peaks > 1 ? kPeakGrid : kMaxGrid);
    void *kargs[] = {&a};
    if (cudaLaunchCooperativeKernel(kfn, grid, kGThreads, kargs, smem, st) !=
        cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    GreedyCtl ctl;
    if (cudaMemcpyAsync(&ctl, ws + L.ctl, kCtlStatBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    *h_nc = ctl.nc;
    if (h_n_hist)
        *h_n_hist = ctl.n_hist;
    if (h_stats) {
        h_stats->iterations = ctl.iterations;
        h_stats->nc = ctl.nc;
        h_stats->full_checks = ctl.full_checks;
        h_stats->pairs_f32 = ctl.pairs_f32;
        h_stats->pairs_f64 = ctl.pairs_f64;
        h_stats->pairs_ff = ctl.pairs_ff;
        h_stats->rescored = (int64_t)ctl.rescored;
        h_stats->estar = ctl.estar;
        h_stats->final_max = ctl.final_max;
        h_stats->final_rms = ctl.final_rms;
        h_stats->min_pivot = ctl.min_pivot;
        h_stats->max_resid = ctl.max_resid;
        for (int i = 0; i < 12; ++i)
            h_stats->phase_ns[i] = (int64_t)ctl.phase_ns[i];
        h_stats->barriers = ctl.barriers;
        h_stats->ctas = grid;
    }
    return (rbf_status)ctl.status;
}

extern "C" rbf_status rbf_greedy_select(const double *d_xb, const double *d_db, int64_t nb,
                                        const rbf_params *p, int32_t *d_sel_idx,
                                        int64_t *d_sel_iter, double *d_w, double *d_hist,
                                        int64_t hist_cap, int64_t *h_nc, int64_t *h_n_hist,
                                        rbf_greedy_stats *h_stats, void *d_ws, size_t ws_bytes,
                                        void *stream)
{
    return greedy_launch(d_xb, d_db, nb, p, d_sel_idx, d_sel_iter, d_w, d_hist, hist_cap, h_nc,
                         h_n_hist, h_stats, d_ws, ws_bytes, stream, 1, 0.0);
}

// ---------------------------------------------------------------------------
// The last stored screened errors and bounds of a greedy workspace, in node
// order, and the weights of the evaluation table (the certified bounds are
// stated for those weights).
// ---------------------------------------------------------------------------
__global__ void k_screen_gather(const int32_t *__restrict__ pos_of_node,
                                const double *__restrict__ e64, const float *__restrict__ u32,
                                int nb, double *__restrict__ e_out, float *__restrict__ b_out)
{
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nb; n += gridDim.x * blockDim.x) {
        const int pos = pos_of_node[n];
        e_out[n] = e64[pos];
        b_out[n] = u32[pos];
    }
}

__global__ void k_table_weights(const float4 *__restrict__ cw32, const float4 *__restrict__ cwff,
                                int prec, int ld, int nc, double *__restrict__ w_out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        double w[3];
        if (prec == RBF_PREC_F32X2) {
            const float4 h = cwff[2 * (size_t)ld + j], l = cwff[3 * (size_t)ld + j];
            w[0] = (double)h.x + (double)l.x;
            w[1] = (double)h.y + (double)l.y;
            w[2] = (double)h.z + (double)l.z;
        } else {
            const float4 h = cw32[(size_t)ld + j];
            w[0] = h.x;
            w[1] = h.y;
            w[2] = h.z;
        }
        for (int c = 0; c < 3; ++c)
            w_out[3 * j + c] = w[c];
    }
}

extern "C" rbf_status rbf_greedy_screen_errors(const void *d_ws, size_t ws_bytes, int64_t nb,
                                               const rbf_params *p, int64_t nc, double *d_err,
                                               float *d_bound, double *d_w_eval, void *stream)
{
    if (!greedy_args_ok(nb, p) || !d_ws || !d_err || !d_bound ||
        (p->eval_prec != RBF_PREC_F32 && p->eval_prec != RBF_PREC_F32X2) || nc < 0 ||
        nc > p->nc_max || (nc > 0 && !d_w_eval))
        return RBF_E_ARG;
    const GreedyWs L = greedy_ws_layout(nb, p->nc_max);
    if (ws_bytes < L.total)
        return RBF_E_WORKSPACE;
    const char *ws = (const char *)d_ws;
    cudaStream_t st = (cudaStream_t)stream;
    k_screen_gather<<<(int)std::min<int64_t>((nb + 255) / 256, 1024), 256, 0, st>>>(
        (const int32_t *)(ws + L.pos_of_node), (const double *)(ws + L.e64),
        (const float *)(ws + L.u32), (int)nb, d_err, d_bound);
    if (nc > 0)
        k_table_weights<<<(int)((nc + 255) / 256), 256, 0, st>>>(
            (const float4 *)(ws + L.cw32), (const float4 *)(ws + L.cwff), p->eval_prec,
            (int)p->nc_max, (int)nc, d_w_eval);
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    return RBF_OK;
}

extern "C" rbf_status rbf_greedy_select_peaks(const double *d_xb, const double *d_db, int64_t nb,
                                              const rbf_params *p, int peaks, double separation,
                                              int32_t *d_sel_idx, int64_t *d_sel_iter,
                                              double *d_w, int64_t *h_nc,
                                              rbf_greedy_stats *h_stats, void *d_ws,
                                              size_t ws_bytes, void *stream)
{
    return greedy_launch(d_xb, d_db, nb, p, d_sel_idx, d_sel_iter, d_w, nullptr, 0, h_nc,
                         nullptr, h_stats, d_ws, ws_bytes, stream, peaks, separation);
}

// ---------------------------------------------------------------------------
// rbf_solve_weights
// ---------------------------------------------------------------------------

extern "C" size_t rbf_solve_workspace_bytes(int64_t nc)
{
    if (nc < 1 || nc > 46340)
        return 0;
    return solve_ws_layout(nc).total;
}

namespace rbf {
static rbf_status solve_launch(const double *d_xb, const double *d_db, int64_t nb,
                               const int32_t *d_sel_idx, int64_t nc, const double *d_rhs,
                               const rbf_params *p, double *d_x, double *h_max_resid, void *d_ws,
                               size_t ws_bytes, void *stream, int reuse = 0)
{
    if (!p || !d_xb || (!d_db && !d_rhs) || !d_sel_idx || !d_x || nc < 1 || nc > nb ||
        nc > 46340 || nb >= kMaxNodes || !(p->radius > 0.0) || !std::isfinite(p->radius) ||
        p->refine_steps < 0 || p->refine_steps > 16)
        return RBF_E_ARG;
    const SolveWs L = solve_ws_layout(nc);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev) || !dev.coop)
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    GreedyArgs a{};
    a.xb = d_xb;
    a.db = d_db;
    a.nb = (int)nb;
    a.m = 1;
    a.nc_max = (int)nc;
    a.prec = RBF_PREC_F64;
    a.inv_r = 1.0 / p->radius;
    a.barrier_ns = kBarrierLimitNs;
    a.ld = (int)nc;
    a.sel_idx = (int32_t *)(ws + L.sel);
    a.sel_iter = nullptr;
    a.hist = nullptr;
    fill_args(a, ws, L.g);
    if (cudaMemsetAsync(ws + L.g.ctl, 0, sizeof(GreedyCtl), st) != cudaSuccess)
        return RBF_E_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve, kGThreads, 0) != cudaSuccess ||
        occ < 1)
        return RBF_E_CUDA;
    // CTAs: a grid barrier costs ~1.1 us among 64 CTAs and 2-3 us among all
    // SMs, while each append's two FP64 matrix-vector products (nc^2 / 2
    // FMAs each) want many SMs once nc passes ~1000
    const int grid = (int)std::min<int64_t>(std::min(dev.sms, kMaxGrid),
                                            std::max<int64_t>(64, nc / 8));
    int nc_i = (int)nc, steps = p->refine_steps;
    D4 *rvec = (D4 *)(ws + L.rvec), *tvec = (D4 *)(ws + L.tvec);
    void *kargs[] = {&a,    (void *)&d_sel_idx, &nc_i, &steps, &rvec, &tvec, &d_x,
                     (void *)&d_rhs, &reuse};
    if (cudaLaunchCooperativeKernel((const void *)k_solve, grid, kGThreads, kargs, 0, st) !=
        cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    GreedyCtl ctl;
    if (cudaMemcpyAsync(&ctl, ws + L.g.ctl, kCtlStatBytes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    if (h_max_resid)
        *h_max_resid = ctl.final_max;
    return (rbf_status)ctl.status;
}
}  // namespace rbf

extern "C" rbf_status rbf_solve_weights(const double *d_xb, const double *d_db, int64_t nb,
                                        const int32_t *d_sel_idx, int64_t nc,
                                        const rbf_params *p, double *d_w, double *h_max_resid,
                                        void *d_ws, size_t ws_bytes, void *stream)
{
    if (!d_db)
        return RBF_E_ARG;
    return solve_launch(d_xb, d_db, nb, d_sel_idx, nc, nullptr, p, d_w, h_max_resid, d_ws,
                        ws_bytes, stream);
}

extern "C" rbf_status rbf_solve_system(const double *d_xb, int64_t nb, const int32_t *d_sel_idx,
                                       int64_t nc, const double *d_rhs, const rbf_params *p,
                                       double *d_x, double *h_max_resid, void *d_ws,
                                       size_t ws_bytes, void *stream)
{
    if (!d_rhs)
        return RBF_E_ARG;
    return solve_launch(d_xb, nullptr, nb, d_sel_idx, nc, d_rhs, p, d_x, h_max_resid, d_ws,
                        ws_bytes, stream);
}

// ---------------------------------------------------------------------------
// Factor objects: the appends of one k_solve launch leave Z = L^-1 of
// Phi_SS in the workspace; later solves with the same support set reuse it.
// ---------------------------------------------------------------------------
extern "C" size_t rbf_factor_workspace_bytes(int64_t nc)
{
    if (nc < 1 || nc > 46340)
        return 0;
    return solve_ws_layout(nc).total + align_up(sizeof(double) * 3 * (size_t)nc, 256);
}

extern "C" rbf_status rbf_factor_create(const double *d_xb, int64_t nb, const int32_t *d_sel_idx,
                                        int64_t nc, const rbf_params *p, void *d_ws,
                                        size_t ws_bytes, void *stream, rbf_factor **out)
{
    if (!out)
        return RBF_E_ARG;
    *out = nullptr;
    if (!p || nc < 1 || nc > 46340)
        return RBF_E_ARG;
    const size_t solve_bytes = solve_ws_layout(nc).total;
    if (!d_ws || ws_bytes < rbf_factor_workspace_bytes(nc) || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    // the appends need a right-hand side: zeros (the factor does not depend on it)
    double *scratch = (double *)((char *)d_ws + solve_bytes);
    if (cudaMemsetAsync(scratch, 0, sizeof(double) * 3 * (size_t)nc, (cudaStream_t)stream) !=
        cudaSuccess)
        return RBF_E_CUDA;
    rbf_params q = *p;
    q.refine_steps = 0;
    const rbf_status st = solve_launch(d_xb, nullptr, nb, d_sel_idx, nc, scratch, &q, scratch,
                                       nullptr, d_ws, solve_bytes, stream, 0);
    if (st != RBF_OK)
        return st;
    rbf_factor *f = new rbf_factor();
    f->xb = d_xb;
    f->nb = nb;
    f->sel = d_sel_idx;
    f->nc = nc;
    f->radius = p->radius;
    f->ws = (char *)d_ws;
    f->ws_bytes = solve_bytes;
    *out = f;
    return RBF_OK;
}

extern "C" rbf_status rbf_factor_solve(const rbf_factor *f, const double *d_rhs, int refine_steps,
                                       double *d_x, double *h_max_resid, void *stream)
{
    if (!f || !d_rhs || !d_x || refine_steps < 0 || refine_steps > 15)
        return RBF_E_ARG;
    rbf_params q{};
    q.radius = f->radius;
    q.refine_steps = refine_steps;
    return solve_launch(f->xb, nullptr, f->nb, f->sel, f->nc, d_rhs, &q, d_x, h_max_resid, f->ws,
                        f->ws_bytes, stream, 1);
}

extern "C" void rbf_factor_destroy(rbf_factor *f) { delete f; }


// ---------------------------------------------------------------------------
// Batched greedy: many independent problems in one cooperative launch.
// ---------------------------------------------------------------------------
struct rbf_greedy_batch {
    int B = 0;
    int grid = 0;
    size_t smem = 0;
    int prec = 0;
    char *ws = nullptr;
    std::vector<size_t> ctl_off;     // control block of each problem (reset per run)
    std::vector<int> cta_start_host; // CTA range of each problem
    size_t args_off = 0, start_off = 0, nc_off = 0;
};

namespace rbf {
struct BatchLayout {
    size_t args, start, nc, total;
    std::vector<size_t> prob;        // workspace segment of each problem
};

static BatchLayout batch_layout(const rbf_greedy_problem *h, int B)
{
    BatchLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.args = take(sizeof(GreedyArgs) * (size_t)B);
    L.start = take(sizeof(int) * (size_t)(B + 1));
    L.nc = take(sizeof(long long) * (size_t)B);
    L.prob.resize(B);
    for (int i = 0; i < B; ++i)
        L.prob[i] = take(greedy_ws_layout(h[i].nb, h[i].params.nc_max).total);
    L.total = o;
    return L;
}
}  // namespace rbf

extern "C" size_t rbf_greedy_batch_workspace_bytes(const rbf_greedy_problem *h_probs, int B)
{
    if (!h_probs || B < 1)
        return 0;
    for (int i = 0; i < B; ++i)
        if (!greedy_args_ok(h_probs[i].nb, &h_probs[i].params))
            return 0;
    return batch_layout(h_probs, B).total;
}

extern "C" rbf_status rbf_greedy_batch_create(const rbf_greedy_problem *h_probs, int B,
                                              void *d_ws, size_t ws_bytes, void *stream,
                                              rbf_greedy_batch **out)
{
    if (!h_probs || B < 1 || !out)
        return RBF_E_ARG;
    *out = nullptr;
    const int prec = h_probs[0].params.eval_prec;
    for (int i = 0; i < B; ++i) {
        const rbf_greedy_problem &q = h_probs[i];
        if (!greedy_args_ok(q.nb, &q.params) || !q.d_xb || !q.d_db || !q.d_sel_idx ||
            q.params.eval_prec != prec || q.params.refine_steps < 0 ||
            q.params.refine_steps > 16 || (q.params.flags & RBF_FLAG_TEST_BARRIER_TIMEOUT))
            return RBF_E_ARG;
    }
    const BatchLayout L = batch_layout(h_probs, B);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    DeviceInfo dev;
    if (!device_info(&dev) || !dev.coop)
        return RBF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    const size_t smem =
        prec == RBF_PREC_F32 ? sizeof(float4) * 2 * kSmemCentresF32
        : prec == RBF_PREC_F32X2 ? sizeof(float4) * 4 * kSmemCentresFF : 0;
    if (cudaFuncSetAttribute(k_greedy_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float4) * 4 * kSmemCentresFF)) != cudaSuccess)
        return RBF_E_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_greedy_batched, kGThreads, smem) !=
            cudaSuccess ||
        occ < 1)
        return RBF_E_CUDA;
    const int total = std::min(dev.sms * std::min(occ, 2), kMaxGrid);
    if (total < B)
        return RBF_E_ARG;   // every problem needs a CTA of its own
    // CTAs: one each, the rest in proportion to the group sizes (the work of
    // one evaluation), capped at 32 per problem
    std::vector<double> wgt(B);
    double wsum = 0.0;
    for (int i = 0; i < B; ++i) {
        wgt[i] = (double)((h_probs[i].nb + h_probs[i].params.m - 1) / h_probs[i].params.m);
        wsum += wgt[i];
    }
    std::vector<int> ctas(B, 1);
    int left = total - B;
    for (int i = 0; i < B && left > 0; ++i) {
        const int extra = std::min(left, std::min(31, (int)(wgt[i] / wsum * (total - B))));
        ctas[i] += extra;
        left -= extra;
    }
    std::vector<int> start(B + 1, 0);
    for (int i = 0; i < B; ++i)
        start[i + 1] = start[i] + ctas[i];
    std::vector<GreedyArgs> args(B);
    for (int i = 0; i < B; ++i) {
        const rbf_greedy_problem &q = h_probs[i];
        const GreedyWs G = greedy_ws_layout(q.nb, q.params.nc_max);
        char *pw = ws + L.prob[i];
        std::vector<int32_t> perm((size_t)q.nb);
        fisher_yates(q.nb, q.params.seed, perm.data());
        if (cudaMemcpyAsync(pw + G.perm, perm.data(), sizeof(int32_t) * q.nb,
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RBF_E_CUDA;
        GreedyArgs &a = args[i];
        a = GreedyArgs{};
        a.xb = q.d_xb;
        a.db = q.d_db;
        a.nb = (int)q.nb;
        a.m = (int)q.params.m;
        a.nc_max = (int)q.params.nc_max;
        a.prec = prec;
        a.inv_r = 1.0 / q.params.radius;
        a.tol = q.params.tol;
        a.tol_mode = q.params.tol_mode;
        a.flags = q.params.flags;
        a.barrier_ns = kBarrierLimitNs;
        a.ld = (int)q.params.nc_max;
        a.sel_idx = q.d_sel_idx;
        a.sel_iter = q.d_sel_iter;
        a.hist = nullptr;
        a.hist_cap = 0;
        a.w_out = q.d_w;
        a.refine_steps = q.params.refine_steps;
        a.smem_cap = (int)std::min<int64_t>(q.params.nc_max, prec == RBF_PREC_F32 ? kSmemCentresF32
                                                             : prec == RBF_PREC_F32X2 ? kSmemCentresFF : 0);
        fill_args(a, pw, G);
        a.nc_out = (long long *)(ws + L.nc) + i;
    }
    if (cudaMemcpyAsync(ws + L.args, args.data(), sizeof(GreedyArgs) * B, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.start, start.data(), sizeof(int) * (B + 1),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RBF_E_CUDA;
    rbf_greedy_batch *b = new rbf_greedy_batch();
    b->B = B;
    b->grid = start[B];
    b->cta_start_host = start;
    b->smem = smem;
    b->prec = prec;
    b->ws = ws;
    b->args_off = L.args;
    b->start_off = L.start;
    b->nc_off = L.nc;
    b->ctl_off.resize(B);
    for (int i = 0; i < B; ++i)
        b->ctl_off[i] = L.prob[i] + greedy_ws_layout(h_probs[i].nb, h_probs[i].params.nc_max).ctl;
    *out = b;
    return RBF_OK;
}

extern "C" rbf_status rbf_greedy_batch_run(rbf_greedy_batch *b, void *stream)
{
    if (!b)
        return RBF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < b->B; ++i)
        if (cudaMemsetAsync(b->ws + b->ctl_off[i], 0, sizeof(GreedyCtl), st) != cudaSuccess)
            return RBF_E_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(kGThreads);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const GreedyArgs *args = (const GreedyArgs *)(b->ws + b->args_off);
    const int *start = (const int *)(b->ws + b->start_off);
    if (cudaLaunchKernelEx(&cfg, k_greedy_batched, args, start, b->B) != cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    return RBF_OK;
}

extern "C" const int64_t *rbf_greedy_batch_nc_device(const rbf_greedy_batch *b)
{
    return b ? (const int64_t *)(b->ws + b->nc_off) : nullptr;
}

extern "C" rbf_status rbf_greedy_batch_results(rbf_greedy_batch *b, int32_t *h_status,
                                               rbf_greedy_stats *h_stats, void *stream)
{
    if (!b)
        return RBF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return RBF_E_CUDA;
    }
    rbf_status worst = RBF_OK;
    for (int i = 0; i < b->B; ++i) {
        GreedyCtl ctl;
        if (cudaMemcpy(&ctl, b->ws + b->ctl_off[i], kCtlStatBytes, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return RBF_E_CUDA;
        if (h_status)
            h_status[i] = ctl.status;
        if (ctl.status != RBF_OK && worst == RBF_OK)
            worst = (rbf_status)ctl.status;
        if (h_stats) {
            rbf_greedy_stats &t = h_stats[i];
            t.iterations = ctl.iterations;
            t.nc = ctl.nc;
            t.full_checks = ctl.full_checks;
            t.pairs_f32 = ctl.pairs_f32;
            t.pairs_f64 = ctl.pairs_f64;
            t.pairs_ff = ctl.pairs_ff;
            t.rescored = (int64_t)ctl.rescored;
            t.estar = ctl.estar;
            t.final_max = ctl.final_max;
            t.final_rms = ctl.final_rms;
            t.min_pivot = ctl.min_pivot;
            t.max_resid = ctl.max_resid;
            for (int k = 0; k < 12; ++k)
                t.phase_ns[k] = (int64_t)ctl.phase_ns[k];
            t.barriers = ctl.barriers;
            t.ctas = b->cta_start_host.empty() ? 0 : b->cta_start_host[i + 1] - b->cta_start_host[i];
        }
    }
    return worst;
}

extern "C" void rbf_greedy_batch_destroy(rbf_greedy_batch *b)
{
    delete b;
}
