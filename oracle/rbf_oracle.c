/*
 * rbf_oracle.c -- plain FP64 CPU oracle for RBF mesh deformation with the
 * grouping-circular-based (GCB) greedy support-node selection.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or helper with the CUDA path, and the product never calls
 * it: only tests/, the smoke check and bench.py's CPU-baseline leg do.
 *
 * Every routine follows the paper step by step, in double precision, with
 * no blocking, fusion or reordering beyond what the text states:
 *
 *   - Wendland C2 basis, Eq. 2:  phi(eta) = (1-eta)^4 (4 eta + 1), eta <= 1;
 *     0 otherwise; eta = distance / R (the "RBF radius", Sec. 2 and Sec. 4).
 *   - RBF interpolant, Eq. 1 and volume displacement, Eq. 6:
 *     F(r) = sum_i w_i phi(|r - r_i| / R), one weight vector per axis, Eq. 4.
 *   - Support system, Eqs. 3-5 restricted to the support set S: Phi_SS W = dX_S,
 *     SPD (Sec. 2), solved by a dense Cholesky factorisation from scratch at
 *     every iteration (the plain re-solve the greedy literature starts from,
 *     Sec. 1).
 *   - GCB greedy, Algorithm 1 (Sec. 3): random uniform partition into m
 *     groups, 3 seed nodes, then for k = 3, 4, ...: solve, i = k mod m,
 *     errors in G_i, local maximum, append if E > E*.
 *
 * Readings of points the paper leaves open:
 *   - error of node q: E_q = || dr_q - F(r_q) ||_2 (Euclidean norm of the
 *     3-vector);
 *   - partition: SplitMix64 stream from the seed, Fisher-Yates shuffle from the
 *     last position down, node perm[p] belongs to group p mod m;
 *   - seed nodes: n0 = argmax |dr|, n1 = farthest node from n0,
 *     n2 = node farthest from {n0, n1}; lowest index on ties;
 *   - argmax ties: lowest node index; nodes already in S are skipped;
 *   - strict comparison E > E*;
 *   - termination: m consecutive iterations that add nothing.  They evaluate
 *     every node once (Sec. 3) with one set of weights, so the global maximum
 *     is then <= E*; the selection sequence is the literal algorithm's.  An
 *     all-node check after every m-th iteration is kept only to fill the
 *     optional error history;
 *   - N_c^max caps |S|.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form phi values, partition
 * invariants, a published SplitMix64 output, brute-force selection on tiny
 * problems through numpy.linalg.solve, reproduction of the prescribed
 * displacement at support nodes, SPD pivots, m = 1 equal to the plain greedy.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_ARG 1
#define ORC_E_NOT_SPD 2
#define ORC_E_NC_MAX 3
#define ORC_E_NOMEM 5
#define ORC_E_FOLLOW 8

/* ------------------------------------------------------------------------ */
/* Eq. 2: Wendland C2 basis function of the normalised distance eta.        */
/* ------------------------------------------------------------------------ */
double orc_phi(double eta)
{
    if (eta > 1.0)
        return 0.0;
    double t = 1.0 - eta;
    return t * t * t * t * (4.0 * eta + 1.0);
}

static double dist3(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* ------------------------------------------------------------------------ */
/* Partition into m groups (Sec. 3, Algorithm 1 first step).               */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): one step of the stream. */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* perm: a random permutation of 0..nb-1 by the Fisher-Yates shuffle driven
 * by SplitMix64(seed).  Node perm[p] is in group p mod m, so the groups are
 * disjoint, cover all nodes and differ in size by at most one. */
void orc_permutation(int64_t nb, uint64_t seed, int32_t *perm)
{
    uint64_t st = seed;
    for (int64_t p = 0; p < nb; ++p)
        perm[p] = (int32_t)p;
    for (int64_t i = nb - 1; i >= 1; --i) {
        uint64_t j = orc_splitmix64_next(&st) % (uint64_t)(i + 1);
        int32_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
}

/* group_of[node] = group index (0..m-1). */
void orc_groups(int64_t nb, int64_t m, uint64_t seed, int32_t *group_of)
{
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
    orc_permutation(nb, seed, perm);
    for (int64_t p = 0; p < nb; ++p)
        group_of[perm[p]] = (int32_t)(p % m);
    free(perm);
}

/* ------------------------------------------------------------------------ */
/* Seed nodes (Algorithm 1: "select any 3 nodes").                          */
/* ------------------------------------------------------------------------ */
void orc_seed_nodes(const double *xb, const double *db, int64_t nb, int32_t out[3])
{
    int64_t n0 = 0;
    double best = -1.0;
    for (int64_t j = 0; j < nb; ++j) {
        const double *d = db + 3 * j;
        double v = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (v > best) { best = v; n0 = j; }
    }
    int64_t n1 = 0;
    best = -1.0;
    for (int64_t j = 0; j < nb; ++j) {
        const double *a = xb + 3 * j, *b = xb + 3 * n0;
        double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
        double v = dx * dx + dy * dy + dz * dz;
        if (v > best) { best = v; n1 = j; }
    }
    int64_t n2 = 0;
    best = -1.0;
    for (int64_t j = 0; j < nb; ++j) {
        const double *a = xb + 3 * j, *b0 = xb + 3 * n0, *b1 = xb + 3 * n1;
        double dx = a[0] - b0[0], dy = a[1] - b0[1], dz = a[2] - b0[2];
        double v0 = dx * dx + dy * dy + dz * dz;
        dx = a[0] - b1[0]; dy = a[1] - b1[1]; dz = a[2] - b1[2];
        double v1 = dx * dx + dy * dy + dz * dz;
        double v = v0 < v1 ? v0 : v1;
        if (v > best) { best = v; n2 = j; }
    }
    out[0] = (int32_t)n0;
    out[1] = (int32_t)n1;
    out[2] = (int32_t)n2;
}

/* ------------------------------------------------------------------------ */
/* Dense SPD solve (Sec. 2: Phi is SPD, so Cholesky applies).               */
/* ------------------------------------------------------------------------ */

/* A squared pivot at or below this fraction of its diagonal entry means the
 * matrix is singular to working precision (coincident nodes make Phi exactly
 * singular, but rounding can leave a pivot of order 1e-16 instead of 0). */
#define ORC_PIVOT_REL 1e-13

/* In-place lower Cholesky of the n x n row-major matrix A (upper part is not
 * referenced).  Returns ORC_E_NOT_SPD if a pivot is not positive. */
int orc_cholesky(int64_t n, double *A)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        double diag = s;
        for (int64_t p = 0; p < j; ++p)
            s -= A[j * n + p] * A[j * n + p];
        if (!(s > ORC_PIVOT_REL * diag))
            return ORC_E_NOT_SPD;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t p = 0; p < j; ++p)
                t -= A[i * n + p] * A[j * n + p];
            A[i * n + j] = t / ljj;
        }
    }
    return ORC_OK;
}

/* Solve L L^T X = B for nrhs right-hand sides stored row-major (n x nrhs). */
void orc_cholesky_solve(int64_t n, const double *L, double *B, int nrhs)
{
    for (int c = 0; c < nrhs; ++c) {
        for (int64_t i = 0; i < n; ++i) {           /* forward: L y = b */
            double t = B[i * nrhs + c];
            for (int64_t p = 0; p < i; ++p)
                t -= L[i * n + p] * B[p * nrhs + c];
            B[i * nrhs + c] = t / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {      /* backward: L^T x = y */
            double t = B[i * nrhs + c];
            for (int64_t p = i + 1; p < n; ++p)
                t -= L[p * n + i] * B[p * nrhs + c];
            B[i * nrhs + c] = t / L[i * n + i];
        }
    }
}

/* Weights of the support set S (Eqs. 4-5 restricted to S): Phi_SS W = dX_S.
 * W is k x 3 row-major.  Optionally returns the smallest Cholesky pivot. */
int orc_solve_weights(const double *xb, const double *db, const int32_t *S, int64_t k,
                      double R, double *W, double *min_pivot)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)(k * k > 0 ? k * k : 1));
    if (!A)
        return ORC_E_NOMEM;
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j)
            A[i * k + j] = orc_phi(dist3(xb + 3 * S[i], xb + 3 * S[j]) / R);
    int st = orc_cholesky(k, A);
    if (st == ORC_OK) {
        for (int64_t i = 0; i < k; ++i)
            for (int c = 0; c < 3; ++c)
                W[i * 3 + c] = db[3 * S[i] + c];
        orc_cholesky_solve(k, A, W, 3);
        if (min_pivot) {
            double mp = INFINITY;
            for (int64_t i = 0; i < k; ++i)
                if (A[i * k + i] < mp) mp = A[i * k + i];
            *min_pivot = mp * mp;
        }
    }
    free(A);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 / Eq. 6: F(r) at arbitrary points, and the interpolation error.    */
/* ------------------------------------------------------------------------ */

/* out (nq x 3) = sum_j W_j phi(|x_q - c_j| / R), centres c_j = xb[S[j]]. */
void orc_rbf_sum(const double *xq, int64_t nq, const double *xb, const int32_t *S,
                 int64_t k, const double *W, double R, double *out, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        double f0 = 0.0, f1 = 0.0, f2 = 0.0;
        for (int64_t j = 0; j < k; ++j) {
            double p = orc_phi(dist3(xq + 3 * q, xb + 3 * S[j]) / R);
            f0 += W[3 * j + 0] * p;
            f1 += W[3 * j + 1] * p;
            f2 += W[3 * j + 2] * p;
        }
        out[3 * q + 0] = f0;
        out[3 * q + 1] = f1;
        out[3 * q + 2] = f2;
    }
    (void)nthreads;
}

/* E_q = |dr_q - F(x_q)|_2 for the listed boundary nodes q = idx[t]. */
static void node_errors(const double *xb, const double *db, const int32_t *idx, int64_t n,
                        const int32_t *S, int64_t k, const double *W, double R,
                        double *E, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t t = 0; t < n; ++t) {
        int32_t q = idx[t];
        double f0 = 0.0, f1 = 0.0, f2 = 0.0;
        for (int64_t j = 0; j < k; ++j) {
            double p = orc_phi(dist3(xb + 3 * q, xb + 3 * S[j]) / R);
            f0 += W[3 * j + 0] * p;
            f1 += W[3 * j + 1] * p;
            f2 += W[3 * j + 2] * p;
        }
        double e0 = db[3 * q + 0] - f0, e1 = db[3 * q + 1] - f1, e2 = db[3 * q + 2] - f2;
        E[t] = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
    }
    (void)nthreads;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: GCB greedy (m = 1 is the plain Rendall-Allen greedy).      */
/* ------------------------------------------------------------------------ */

/* History rows: [iteration k, |S| before the step, local max E in G_i,
 *                global max E (or -1 if no full check), global RMS E (or -1),
 *                added node (or -1)].  */
#define ORC_HIST_COLS 6

typedef struct {
    int64_t iterations;   /* iterations run (k - 3 at exit)                 */
    int64_t full_checks;  /* number of all-node error evaluations           */
    int64_t pairs_group;  /* sum over iterations of |G_i| * |S| (Sec. 3)    */
    int64_t pairs_full;   /* sum over full checks of N_b * |S|              */
    double final_max;     /* global max E at exit (current weights)        */
    double final_rms;
    double min_pivot;     /* smallest Cholesky pivot seen (SPD check)       */
    int64_t n_div;        /* follow mode: accepted divergences              */
    int64_t n_fail;       /* follow mode: rejected steps                    */
    double worst_rel_gap; /* follow mode: largest relative gap of any checked
                           * decision: (max E - E_follow)/max E for an append,
                           * (E* - E_follow)/E* for an append at or below E*,
                           * (max E - E*)/E* for "no add" above E*           */
} orc_greedy_stats;

/*
 * follow mode (follow_n >= 0): instead of adding its own argmax, the oracle
 * adopts the decision of another implementation, given as the nodes it added
 * (follow_idx) and the iteration at which each was added (follow_iter).  At
 * every iteration it checks that decision against its own FP64 errors:
 *   - an added node must lie in G_i, not be in S, have E > E*(1 - tie) and
 *     E >= (1 - tie) * max_G_i E; it counts as a divergence when it is not
 *     the oracle's own argmax or when its E is not above E* (the literal
 *     algorithm would not have appended it);
 *   - "no add" is accepted when max_G_i E <= E*(1 + tie), and counts as a
 *     divergence when max_G_i E > E*.
 * The 1e-6 band of the comparison is relative: both the argmax and the
 * E > E* test may go the other way only where the two values compared agree
 * to tie_rel; each such step is counted in n_div and its gap in
 * worst_rel_gap.
 * follow_n < 0 runs the literal algorithm.
 */
int orc_greedy(const double *xb, const double *db, int64_t nb, double R, double Estar,
               int64_t m, uint64_t seed, int64_t ncmax,
               const int32_t *follow_idx, const int64_t *follow_iter, int64_t follow_n,
               double tie_rel,
               int32_t *out_idx, int64_t *out_iter, int64_t *out_nc,
               double *hist, int64_t hist_cap, int64_t *n_hist,
               orc_greedy_stats *stats, int nthreads)
{
    if (nb < 3 || m < 1 || m > nb || ncmax < 3 || !(R > 0.0) || !(Estar >= 0.0))
        return ORC_E_ARG;
    memset(stats, 0, sizeof(*stats));
    stats->min_pivot = INFINITY;
    int32_t *group_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int64_t *goff = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    char *inS = (char *)calloc((size_t)nb, 1);
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    double *E = (double *)malloc(sizeof(double) * (size_t)nb);
    double *W = (double *)malloc(sizeof(double) * 3 * (size_t)ncmax);
    if (!group_of || !members || !goff || !inS || !all || !E || !W) {
        free(group_of); free(members); free(goff); free(inS); free(all); free(E); free(W);
        return ORC_E_NOMEM;
    }
    /* Step 1: partition; members of each group listed in node order. */
    orc_groups(nb, m, seed, group_of);
    for (int64_t j = 0; j < nb; ++j)
        goff[group_of[j] + 1]++;
    for (int64_t g = 0; g < m; ++g)
        goff[g + 1] += goff[g];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        for (int64_t g = 0; g < m; ++g)
            fill[g] = goff[g];
        for (int64_t j = 0; j < nb; ++j)
            members[fill[group_of[j]]++] = (int32_t)j;
        free(fill);
    }
    for (int64_t j = 0; j < nb; ++j)
        all[j] = (int32_t)j;

    /* Step 2: three seed nodes. */
    int32_t seeds[3];
    orc_seed_nodes(xb, db, nb, seeds);
    int64_t nc = 0;
    for (int s = 0; s < 3; ++s) {
        out_idx[nc] = seeds[s];
        out_iter[nc] = -1;
        inS[seeds[s]] = 1;
        ++nc;
    }
    int64_t fpos = 0;
    if (follow_n >= 0) {
        /* the follower must start from the same seed nodes */
        for (int s = 0; s < 3; ++s)
            if (follow_n <= s || follow_idx[s] != seeds[s])
                stats->n_fail++;
        fpos = 3;
    }
    int status = ORC_OK;
    int64_t nh = 0;
    int64_t idle = 0;          /* consecutive iterations without an append */
    double run_max = 0.0, run_sq = 0.0;
    int64_t k = 3;
    for (;; ++k) {
        /* Solve Phi_SS W = dX_S from scratch (dense Cholesky). */
        double mp;
        int st = orc_solve_weights(xb, db, out_idx, nc, R, W, &mp);
        if (st != ORC_OK) { status = st; break; }
        if (mp < stats->min_pivot) stats->min_pivot = mp;

        /* i = k mod m; errors in G_i (nodes already in S are skipped). */
        int64_t gi = k % m;
        int64_t g0 = goff[gi], gn = goff[gi + 1] - goff[gi];
        node_errors(xb, db, members + g0, gn, out_idx, nc, W, R, E, nthreads);
        stats->pairs_group += gn * nc;
        double Eloc = -1.0;
        int64_t nloc = -1;
        for (int64_t t = 0; t < gn; ++t) {
            int32_t q = members[g0 + t];
            if (inS[q]) continue;
            if (E[t] > Eloc) { Eloc = E[t]; nloc = q; }   /* ascending q: lowest index wins ties */
        }
        int64_t add = -1;
        if (follow_n < 0) {
            if (nloc >= 0 && Eloc > Estar)
                add = nloc;
        } else {
            int follower_adds = (fpos < follow_n && follow_iter[fpos] == k);
            if (follower_adds) {
                int32_t nf = follow_idx[fpos];
                double Ef = -1.0;
                int ok = nf >= 0 && nf < nb && group_of[nf] == gi && !inS[nf];
                if (ok) {
                    for (int64_t t = 0; t < gn; ++t)
                        if (members[g0 + t] == nf) { Ef = E[t]; break; }
                    ok = Ef > Estar * (1.0 - tie_rel) && Ef >= (1.0 - tie_rel) * Eloc;
                }
                if (!ok) stats->n_fail++;
                else if (nf != nloc || !(Ef > Estar)) stats->n_div++;
                if (Eloc > 0.0 && Ef >= 0.0) {
                    double gap = (Eloc - Ef) / Eloc;
                    if (gap > stats->worst_rel_gap) stats->worst_rel_gap = gap;
                }
                if (Estar > 0.0 && Ef >= 0.0 && !(Ef > Estar)) {
                    double gap = (Estar - Ef) / Estar;
                    if (gap > stats->worst_rel_gap) stats->worst_rel_gap = gap;
                }
                add = nf;
                fpos++;
            } else {
                /* the followed run is used up and stopped at its capacity:
                 * this is the iteration where the literal algorithm would
                 * append beyond N_c^max */
                if (fpos >= follow_n && nc >= ncmax && nloc >= 0 && Eloc > Estar) {
                    status = ORC_E_NC_MAX;
                    break;
                }
                if (nloc >= 0 && Eloc > Estar * (1.0 + tie_rel)) stats->n_fail++;
                else if (nloc >= 0 && Eloc > Estar) stats->n_div++;
                if (nloc >= 0 && Estar > 0.0 && Eloc > Estar) {
                    double gap = (Eloc - Estar) / Estar;
                    if (gap > stats->worst_rel_gap) stats->worst_rel_gap = gap;
                }
            }
        }
        if (add >= 0) {
            if (nc >= ncmax) {
                status = ORC_E_NC_MAX;
                break;
            }
            out_idx[nc] = (int32_t)add;
            out_iter[nc] = k;
            inS[add] = 1;
            ++nc;
        }
        /* Termination (Sec. 3: after m iterations every boundary node has had
         * its error computed once): m consecutive iterations that add nothing
         * evaluated every node with the same weights and found E <= E*. */
        if (add >= 0) {
            idle = 0;
            run_max = 0.0;
            run_sq = 0.0;
        } else {
            ++idle;
            for (int64_t t = 0; t < gn; ++t) {
                if (E[t] > run_max) run_max = E[t];
                run_sq += E[t] * E[t];
            }
        }
        /* Optional history: all-node errors after every m-th iteration. */
        int full = hist != NULL && ((k - 2) % m == 0);
        double gmax = -1.0, grms = -1.0;
        if (full) {
            if (add >= 0) {
                st = orc_solve_weights(xb, db, out_idx, nc, R, W, &mp);
                if (st != ORC_OK) { status = st; break; }
                if (mp < stats->min_pivot) stats->min_pivot = mp;
            }
            node_errors(xb, db, all, nb, out_idx, nc, W, R, E, nthreads);
            stats->full_checks++;
            stats->pairs_full += nb * nc;
            double s2 = 0.0;
            gmax = 0.0;
            for (int64_t j = 0; j < nb; ++j) {
                if (E[j] > gmax) gmax = E[j];
                s2 += E[j] * E[j];
            }
            grms = sqrt(s2 / (double)nb);
        }
        if (hist && nh < hist_cap) {
            double *h = hist + ORC_HIST_COLS * nh;
            h[0] = (double)k;
            h[1] = (double)(add >= 0 ? nc - 1 : nc);
            h[2] = Eloc;
            h[3] = gmax;
            h[4] = grms;
            h[5] = (double)add;
        }
        ++nh;
        if (idle >= m) {
            stats->final_max = run_max;
            stats->final_rms = sqrt(run_sq / (double)nb);
            break;
        }
    }
    if (follow_n >= 0 && fpos != follow_n)
        stats->n_fail++;
    stats->iterations = k - 3 + 1;
    *out_nc = nc;
    *n_hist = nh;
    free(group_of); free(members); free(goff); free(inS); free(all); free(E); free(W);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of Eq. 6 for J(d_v) with d_v = Phi_vc W, W = Phi_cc^{-1} d_c:     */
/*   dJ/dd_c = Phi_cc^{-1} Phi_vc^T dJ/dd_v  (Phi_cc symmetric).            */
/* ------------------------------------------------------------------------ */
int orc_adjoint(const double *xv, int64_t nv, const double *xb, const int32_t *S, int64_t k,
                double R, const double *gv, double *gc, int nthreads)
{
    /* g = Phi_vc^T gv, accumulated column by column in fixed order */
    for (int64_t j = 0; j < k; ++j) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t v = 0; v < nv; ++v) {
            double p = orc_phi(dist3(xv + 3 * v, xb + 3 * S[j]) / R);
            a0 += p * gv[3 * v + 0];
            a1 += p * gv[3 * v + 1];
            a2 += p * gv[3 * v + 2];
        }
        gc[3 * j + 0] = a0;
        gc[3 * j + 1] = a1;
        gc[3 * j + 2] = a2;
    }
    (void)nthreads;
    /* solve Phi_cc lambda = g */
    double *A = (double *)malloc(sizeof(double) * (size_t)(k * k > 0 ? k * k : 1));
    if (!A)
        return ORC_E_NOMEM;
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j)
            A[i * k + j] = orc_phi(dist3(xb + 3 * S[i], xb + 3 * S[j]) / R);
    int st = orc_cholesky(k, A);
    if (st == ORC_OK)
        orc_cholesky_solve(k, A, gc, 3);
    free(A);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Peak-selection variant (prior art cited in Sec. 1: several error-peak     */
/* nodes added at a time).  Reading: in iteration k the nodes of G_(k mod m) */
/* outside S with E > E* are taken in decreasing E (lowest index on ties),   */
/* each only if it lies at least `sep` from every node already taken in this */
/* iteration, up to `peaks` nodes; they are appended in that order.  peaks   */
/* = 1 is Algorithm 1.  Termination as orc_greedy: m consecutive iterations  */
/* without an append.  Literal algorithm only (no follow mode, no history).  */
/* ------------------------------------------------------------------------ */
int orc_greedy_peaks(const double *xb, const double *db, int64_t nb, double R, double Estar,
                     int64_t m, uint64_t seed, int64_t ncmax, int64_t peaks, double sep,
                     int32_t *out_idx, int64_t *out_iter, int64_t *out_nc,
                     int64_t *out_iterations, int nthreads)
{
    if (nb < 3 || m < 1 || m > nb || ncmax < 3 || !(R > 0.0) || !(Estar >= 0.0) || peaks < 1 ||
        !(sep >= 0.0))
        return ORC_E_ARG;
    int32_t *group_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int64_t *goff = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    char *inS = (char *)calloc((size_t)nb, 1);
    char *used = (char *)calloc((size_t)nb, 1);
    double *E = (double *)malloc(sizeof(double) * (size_t)nb);
    double *W = (double *)malloc(sizeof(double) * 3 * (size_t)ncmax);
    int32_t *taken = (int32_t *)malloc(sizeof(int32_t) * (size_t)peaks);
    if (!group_of || !members || !goff || !inS || !used || !E || !W || !taken) {
        free(group_of); free(members); free(goff); free(inS); free(used); free(E); free(W);
        free(taken);
        return ORC_E_NOMEM;
    }
    /* partition and seed nodes exactly as orc_greedy */
    orc_groups(nb, m, seed, group_of);
    for (int64_t j = 0; j < nb; ++j)
        goff[group_of[j] + 1]++;
    for (int64_t g = 0; g < m; ++g)
        goff[g + 1] += goff[g];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        for (int64_t g = 0; g < m; ++g)
            fill[g] = goff[g];
        for (int64_t j = 0; j < nb; ++j)
            members[fill[group_of[j]]++] = (int32_t)j;
        free(fill);
    }
    int32_t seeds[3];
    orc_seed_nodes(xb, db, nb, seeds);
    int64_t nc = 0;
    for (int s = 0; s < 3; ++s) {
        out_idx[nc] = seeds[s];
        out_iter[nc] = -1;
        inS[seeds[s]] = 1;
        ++nc;
    }
    int status = ORC_OK;
    int64_t idle = 0, k = 3;
    for (;; ++k) {
        double mp;
        int st = orc_solve_weights(xb, db, out_idx, nc, R, W, &mp);
        if (st != ORC_OK) { status = st; break; }
        int64_t gi = k % m;
        int64_t g0 = goff[gi], gn = goff[gi + 1] - goff[gi];
        node_errors(xb, db, members + g0, gn, out_idx, nc, W, R, E, nthreads);
        /* take peaks: largest E first, separated by at least sep */
        int64_t nt = 0;
        for (int64_t r = 0; r < peaks; ++r) {
            double best = -1.0;
            int64_t bt = -1;
            for (int64_t t = 0; t < gn; ++t) {
                int32_t q = members[g0 + t];
                if (inS[q] || used[q] || !(E[t] > Estar) || !(E[t] > best))
                    continue;   /* ascending q: the lowest index wins ties */
                int far = 1;
                for (int64_t u = 0; u < nt; ++u)
                    if (dist3(xb + 3 * q, xb + 3 * taken[u]) < sep) { far = 0; break; }
                if (far) { best = E[t]; bt = t; }
            }
            if (bt < 0)
                break;
            taken[nt++] = members[g0 + bt];
            used[members[g0 + bt]] = 1;
        }
        for (int64_t u = 0; u < nt; ++u)
            used[taken[u]] = 0;
        if (nt == 0) {
            if (++idle >= m)
                break;
            continue;
        }
        idle = 0;
        for (int64_t u = 0; u < nt; ++u) {
            if (nc >= ncmax) { status = ORC_E_NC_MAX; break; }
            out_idx[nc] = taken[u];
            out_iter[nc] = k;
            inS[taken[u]] = 1;
            ++nc;
        }
        if (status != ORC_OK)
            break;
    }
    *out_nc = nc;
    *out_iterations = k - 3 + 1;
    free(group_of); free(members); free(goff); free(inS); free(used); free(E); free(W);
    free(taken);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Kullback-Leibler divergence of two support sets (Sec. 4.1):              */
/*   KL(S1 || S2) = sum_{i=1..N_b} d1_i log(d1_i / d2_i),                     */
/*   dk_i = min over j in Sk of |r_i - r_j|  (every boundary node i).        */
/* The paper is silent on d = 0 (node i belongs to a set): such terms have   */
/* no finite logarithm and are left out.  The sum runs in node order.        */
/* ------------------------------------------------------------------------ */
void orc_nearest_support(const double *xb, int64_t nb, const int32_t *S, int64_t k,
                         double *d, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t i = 0; i < nb; ++i) {
        double best = INFINITY;
        for (int64_t j = 0; j < k; ++j) {
            double dij = dist3(xb + 3 * i, xb + 3 * S[j]);
            if (dij < best)
                best = dij;
        }
        d[i] = best;
    }
    (void)nthreads;
}

int orc_support_kl(const double *xb, int64_t nb, const int32_t *S1, int64_t k1,
                   const int32_t *S2, int64_t k2, double *kl, int nthreads)
{
    double *d1 = (double *)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    double *d2 = (double *)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    if (!d1 || !d2) {
        free(d1);
        free(d2);
        return ORC_E_NOMEM;
    }
    orc_nearest_support(xb, nb, S1, k1, d1, nthreads);
    orc_nearest_support(xb, nb, S2, k2, d2, nthreads);
    double sum = 0.0;
    for (int64_t i = 0; i < nb; ++i)
        if (d1[i] > 0.0 && d2[i] > 0.0)
            sum += d1[i] * log(d1[i] / d2[i]);
    *kl = sum;
    free(d1);
    free(d2);
    return ORC_OK;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* cpu_rc: Algorithm 1 with the recurrence Cholesky (RC) decomposition of   */
/* Sec. 1 and Table 1 instead of a dense re-solve -- the paper's own CPU     */
/* procedure, kept as the fair CPU baseline of the timings.  Appending node  */
/* n to S grows the lower Cholesky factor L of Phi_SS by one row:            */
/*   b_j = phi(|r_n - r_j| / R) (j in S),  L l = b (forward substitution),   */
/*   d = sqrt(phi(0) - l.l),  new row [l^T, d],                              */
/* and the forward vector y (L y = dX_S) by y_n = (dr_n - l.y) / d; the      */
/* weights then follow from L^T W = y (back substitution).  FP64 throughout; */
/* the group errors are evaluated in parallel over nodes.  out_w (nullable, */
/* ncmax x 3) receives the final weights.  Partition, seed                   */
/* nodes, argmax, E > E* and termination are those of orc_greedy, so the two */
/* select the same sequence unless rounding separates two near-equal errors. */
/* A squared pivot d^2 <= 1e-13 (of phi(0) = 1) is singular (ORC_E_NOT_SPD). */
/* ------------------------------------------------------------------------ */
int orc_greedy_rc(const double *xb, const double *db, int64_t nb, double R, double Estar,
                  int64_t m, uint64_t seed, int64_t ncmax,
                  int32_t *out_idx, int64_t *out_iter, int64_t *out_nc,
                  int64_t *out_iterations, double *final_max, double *out_w, int nthreads)
{
    if (nb < 3 || m < 1 || m > nb || ncmax < 3 || !(R > 0.0) || !(Estar >= 0.0))
        return ORC_E_ARG;
    int32_t *group_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int64_t *goff = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    char *inS = (char *)calloc((size_t)nb, 1);
    double *E = (double *)malloc(sizeof(double) * (size_t)nb);
    double *W = (double *)malloc(sizeof(double) * 3 * (size_t)ncmax);
    double *Y = (double *)malloc(sizeof(double) * 3 * (size_t)ncmax);
    double *L = (double *)malloc(sizeof(double) * (size_t)ncmax * (size_t)ncmax);
    double *l = (double *)malloc(sizeof(double) * (size_t)ncmax);
    if (!group_of || !members || !goff || !inS || !E || !W || !Y || !L || !l) {
        free(group_of); free(members); free(goff); free(inS); free(E); free(W); free(Y);
        free(L); free(l);
        return ORC_E_NOMEM;
    }
    orc_groups(nb, m, seed, group_of);
    for (int64_t j = 0; j < nb; ++j)
        goff[group_of[j] + 1]++;
    for (int64_t g = 0; g < m; ++g)
        goff[g + 1] += goff[g];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        for (int64_t g = 0; g < m; ++g)
            fill[g] = goff[g];
        for (int64_t j = 0; j < nb; ++j)
            members[fill[group_of[j]]++] = (int32_t)j;
        free(fill);
    }
    int status = ORC_OK;
    int64_t nc = 0;
    /* RC append of node n as row nc of L (row-major, leading dimension ncmax) */
#define RC_APPEND(n_, it_)                                                       \
    do {                                                                         \
        const int32_t nn = (n_);                                                 \
        double ll = 0.0, ly0 = 0.0, ly1 = 0.0, ly2 = 0.0;                        \
        for (int64_t i = 0; i < nc; ++i) {                                       \
            double t = orc_phi(dist3(xb + 3 * nn, xb + 3 * out_idx[i]) / R);     \
            for (int64_t p = 0; p < i; ++p)                                      \
                t -= L[i * ncmax + p] * l[p];                                    \
            l[i] = t / L[i * ncmax + i];                                         \
            ll += l[i] * l[i];                                                   \
            ly0 += l[i] * Y[3 * i + 0];                                          \
            ly1 += l[i] * Y[3 * i + 1];                                          \
            ly2 += l[i] * Y[3 * i + 2];                                          \
        }                                                                        \
        const double d2 = orc_phi(0.0) - ll;                                     \
        if (!(d2 > ORC_PIVOT_REL)) { status = ORC_E_NOT_SPD; break; }            \
        const double d = sqrt(d2);                                               \
        for (int64_t p = 0; p < nc; ++p)                                         \
            L[nc * ncmax + p] = l[p];                                            \
        L[nc * ncmax + nc] = d;                                                  \
        Y[3 * nc + 0] = (db[3 * nn + 0] - ly0) / d;                              \
        Y[3 * nc + 1] = (db[3 * nn + 1] - ly1) / d;                              \
        Y[3 * nc + 2] = (db[3 * nn + 2] - ly2) / d;                              \
        out_idx[nc] = nn;                                                        \
        out_iter[nc] = (it_);                                                    \
        inS[nn] = 1;                                                             \
        ++nc;                                                                    \
    } while (0)

    int32_t seeds[3];
    orc_seed_nodes(xb, db, nb, seeds);
    for (int s = 0; s < 3 && status == ORC_OK; ++s)
        RC_APPEND(seeds[s], -1);
    int64_t idle = 0, k = 3;
    double run_max = 0.0;
    int stale = 1;   /* W must be recomputed from L and y */
    for (; status == ORC_OK; ++k) {
        if (stale) {
            /* back substitution L^T W = y */
            for (int64_t i = nc - 1; i >= 0; --i)
                for (int c = 0; c < 3; ++c) {
                    double t = Y[3 * i + c];
                    for (int64_t p = i + 1; p < nc; ++p)
                        t -= L[p * ncmax + i] * W[3 * p + c];
                    W[3 * i + c] = t / L[i * ncmax + i];
                }
            stale = 0;
        }
        int64_t gi = k % m;
        int64_t g0 = goff[gi], gn = goff[gi + 1] - goff[gi];
        node_errors(xb, db, members + g0, gn, out_idx, nc, W, R, E, nthreads);
        double Eloc = -1.0;
        int64_t nloc = -1;
        for (int64_t t = 0; t < gn; ++t) {
            int32_t q = members[g0 + t];
            if (inS[q]) continue;
            if (E[t] > Eloc) { Eloc = E[t]; nloc = q; }
        }
        if (nloc >= 0 && Eloc > Estar) {
            if (nc >= ncmax) { status = ORC_E_NC_MAX; break; }
            RC_APPEND((int32_t)nloc, k);
            stale = 1;
            idle = 0;
            run_max = 0.0;
        } else {
            for (int64_t t = 0; t < gn; ++t)
                if (E[t] > run_max) run_max = E[t];
            if (++idle >= m)
                break;
        }
    }
#undef RC_APPEND
    if (out_w && status == ORC_OK) {
        /* final weights of the selected set: L^T W = y */
        for (int64_t i = nc - 1; i >= 0; --i)
            for (int c = 0; c < 3; ++c) {
                double t = Y[3 * i + c];
                for (int64_t p = i + 1; p < nc; ++p)
                    t -= L[p * ncmax + i] * out_w[3 * p + c];
                out_w[3 * i + c] = t / L[i * ncmax + i];
            }
    }
    *out_nc = nc;
    *out_iterations = k - 3 + 1;
    *final_max = run_max;
    free(group_of); free(members); free(goff); free(inS); free(E); free(W); free(Y);
    free(L); free(l);
    return status;
}
